// Lockstep batching of the iterative solves of several RVEs of one grid (host side).
//
// Each RVE keeps its own engine, buffers, stream and host control (the staggered loop, the
// control search, Anderson mixing), run in a host thread of its own. When a thread reaches the
// iteration loop of a solve (the equilibrium CG or the damage PCG), it hands the loop to the
// Batcher as a LoopReq and waits. The Batcher's coordinator groups the loops it holds by kind and
// runs them as batched launches: one kernel launch per pass serves every RVE of a kind
// (blockIdx.z selects the RVE), one chunk of iterations at a time; after each chunk it releases
// the loops whose own scalar block says done and admits the loops that have arrived. An RVE that
// has converged skips its share of the work (its kernels test its done flag), so each RVE
// performs exactly the iterations it would perform alone, with the same arithmetic and the same
// reduction order: its results are bit-identical to stepping it alone.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "pff_common.cuh"
#include "pff_kernels.cuh"

namespace pffeng {

using pff::Scal;
using pff::kMaxBatch;

struct LoopReq {
    // runs `iters` batched iterations of the group (all members share this function)
    void (*launch)(std::vector<LoopReq *> &grp, cudaStream_t st, int iters) = nullptr;
    Scal *sc = nullptr;        // the RVE's device scalars
    Scal *h_sc = nullptr;      // pinned host copy, filled when the loop has finished
    cudaStream_t slot_stream = nullptr;
    cudaEvent_t ready = nullptr, finished = nullptr;
    long *launch_counter = nullptr;
    bool done = false;
    cudaError_t err = cudaSuccess;
    virtual ~LoopReq() {}
};

class Batcher {
  public:
    // When no loop is active, the first chunk waits for company. window_us < 0: until every
    // participant is waiting or done (participants that advance together, as in rve_step_batch);
    // window_us >= 0: at most that long after the first loop arrived (participants that advance
    // independently, as in the request server, then do not stall on one another's host work).
    // While loops are active, new ones join at the next chunk.
    explicit Batcher(int device, int chunk = 8, double window_us = -1.0)
        : device_(device), chunk_(chunk), window_us_(window_us) {
        cudaSetDevice(device_);
        err_ = cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking);
        coord_ = std::thread([this] { loop(); });
    }
    ~Batcher() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_coord_.notify_all();
        coord_.join();
        if (st_) cudaStreamDestroy(st_);
    }
    Batcher(const Batcher &) = delete;
    Batcher &operator=(const Batcher &) = delete;
    cudaError_t status() const { return err_; }
    long batched_launches() const { return launches_; }
    int max_group() const { return max_group_; }

    // A participant starts (before its thread runs) / finishes.
    void join() {
        std::lock_guard<std::mutex> lk(mu_);
        ++running_;
    }
    void leave() {
        std::lock_guard<std::mutex> lk(mu_);
        --running_;
        cv_coord_.notify_all();
    }
    // Hand one iteration loop over and wait until it has run. On return the request's h_sc holds
    // the final scalars and the slot stream is ordered after the batched work.
    void run(LoopReq *r) {
        r->err = cudaEventRecord(r->ready, r->slot_stream);
        {
            std::unique_lock<std::mutex> lk(mu_);
            r->done = false;
            if (waiting_.empty()) first_wait_ = std::chrono::steady_clock::now();
            waiting_.push_back(r);
            --running_;
            cv_coord_.notify_all();
            cv_slots_.wait(lk, [&] { return r->done; });
            ++running_;
        }
        if (r->err == cudaSuccess) r->err = cudaStreamWaitEvent(r->slot_stream, r->finished, 0);
    }

  private:
    // Continuous batching at chunk granularity: the coordinator keeps a set of active loops,
    // admits the loops that arrived while the previous chunk ran, launches one chunk of
    // iterations for every active loop (one launch per pass and kind, up to kMaxBatch RVEs per
    // launch), reads every active loop's scalars back, and releases the loops that are done, so
    // that a loop that converges early does not wait for the slowest one and a loop that
    // arrives late does not wait for the running ones to finish. A loop's arithmetic does not
    // depend on which other loops share its launches, so where it joins does not change its bits.
    void loop() {
        cudaSetDevice(device_);
        std::vector<LoopReq *> active;
        for (;;) {
            std::vector<LoopReq *> fresh;
            {
                std::unique_lock<std::mutex> lk(mu_);
                if (active.empty()) {
                    if (window_us_ < 0.0) {
                        cv_coord_.wait(lk, [&] { return stop_ || (running_ == 0 && !waiting_.empty()); });
                    } else {
                        cv_coord_.wait(lk, [&] { return stop_ || !waiting_.empty(); });
                        if (!waiting_.empty()) {
                            const auto until = first_wait_ + std::chrono::microseconds((long)window_us_);
                            cv_coord_.wait_until(lk, until, [&] { return stop_ || running_ == 0; });
                        }
                    }
                    if (waiting_.empty()) return;  // stop requested and nothing left
                }
                fresh.swap(waiting_);
            }
            cudaError_t e = cudaSuccess;
            for (LoopReq *r : fresh) {
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st_, r->ready, 0);
                active.push_back(r);
            }
            if (e == cudaSuccess) e = chunk(active);
            // release the loops that are done (all of them after an error)
            std::vector<LoopReq *> keep;
            bool released = false;
            for (LoopReq *r : active) {
                if (e != cudaSuccess || r->h_sc->done) {
                    cudaError_t f = e;
                    if (f == cudaSuccess) f = cudaEventRecord(r->finished, st_);
                    r->err = f;
                    std::lock_guard<std::mutex> lk(mu_);
                    r->done = true;
                    released = true;
                } else {
                    keep.push_back(r);
                }
            }
            active.swap(keep);
            if (released) cv_slots_.notify_all();
        }
    }
    // One chunk of iterations for every active loop, then their scalars on the host.
    cudaError_t chunk(std::vector<LoopReq *> &active) {
        std::map<void *, std::vector<LoopReq *>> kinds;
        for (LoopReq *r : active) kinds[(void *)r->launch].push_back(r);
        cudaError_t e = cudaSuccess;
        for (auto &kv : kinds) {
            std::vector<LoopReq *> &all = kv.second;
            for (size_t b0 = 0; b0 < all.size() && e == cudaSuccess; b0 += kMaxBatch) {
                std::vector<LoopReq *> grp(all.begin() + b0, all.begin() + std::min(all.size(), b0 + kMaxBatch));
                max_group_ = std::max(max_group_, (int)grp.size());
                grp[0]->launch(grp, st_, chunk_);
                launches_ += chunk_;
                e = cudaGetLastError();
            }
        }
        for (LoopReq *r : active)
            if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_sc, r->sc, sizeof(Scal), cudaMemcpyDeviceToHost, st_);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
        return e;
    }

    int device_;
    int chunk_;
    double window_us_;
    std::chrono::steady_clock::time_point first_wait_;
    cudaStream_t st_ = nullptr;
    cudaError_t err_ = cudaSuccess;
    std::mutex mu_;
    std::condition_variable cv_coord_, cv_slots_;
    int running_ = 0;
    bool stop_ = false;
    std::vector<LoopReq *> waiting_;
    std::thread coord_;
    long launches_ = 0;
    int max_group_ = 0;
};

}  // namespace pffeng
