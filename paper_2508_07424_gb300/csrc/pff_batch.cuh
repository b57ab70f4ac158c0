// Lockstep batching of the iterative solves of several RVEs of one grid (host side).
//
// Each RVE keeps its own engine, buffers, stream and host control (the staggered loop, the
// control search, Anderson mixing), run in a host thread of its own. When a thread reaches the
// iteration loop of a solve (the equilibrium CG or the damage PCG), it hands the loop to the
// Batcher as a LoopReq and waits. Once every participating thread is either waiting or done, the
// Batcher's coordinator groups the waiting loops by kind and runs each group as batched
// launches: one kernel launch per pass serves every RVE of the group (blockIdx.z selects the
// RVE), in chunks of iterations, until every RVE's own scalar block says done. An RVE that has
// converged skips its share of the work (its kernels test its done flag), so each RVE performs
// exactly the iterations it would perform alone, with the same arithmetic and the same reduction
// order: its results are bit-identical to stepping it alone.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
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
    explicit Batcher(int device, int chunk = 8) : device_(device), chunk_(chunk) {
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
            waiting_.push_back(r);
            --running_;
            cv_coord_.notify_all();
            cv_slots_.wait(lk, [&] { return r->done; });
            ++running_;
        }
        if (r->err == cudaSuccess) r->err = cudaStreamWaitEvent(r->slot_stream, r->finished, 0);
    }

  private:
    void loop() {
        cudaSetDevice(device_);
        for (;;) {
            std::vector<LoopReq *> batch;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_coord_.wait(lk, [&] { return stop_ || (running_ == 0 && !waiting_.empty()); });
                if (waiting_.empty()) return;  // stop requested and nothing left
                batch.swap(waiting_);
            }
            execute(batch);
            {
                std::lock_guard<std::mutex> lk(mu_);
                for (LoopReq *r : batch) r->done = true;
            }
            cv_slots_.notify_all();
        }
    }
    void execute(std::vector<LoopReq *> &batch) {
        // group by kind (launch function), at most kMaxBatch RVEs per launch
        std::map<void *, std::vector<LoopReq *>> kinds;
        for (LoopReq *r : batch) kinds[(void *)r->launch].push_back(r);
        for (auto &kv : kinds) {
            std::vector<LoopReq *> &all = kv.second;
            for (size_t b0 = 0; b0 < all.size(); b0 += kMaxBatch) {
                std::vector<LoopReq *> grp(all.begin() + b0, all.begin() + std::min(all.size(), b0 + kMaxBatch));
                cudaError_t e = cudaSuccess;
                for (LoopReq *r : grp)
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(st_, r->ready, 0);
                max_group_ = std::max(max_group_, (int)grp.size());
                // chunks of iterations until every member is done (each member's kernels stop
                // working once its own done flag is set; its iteration cap sets it at the latest)
                for (int guard = 0; e == cudaSuccess; ++guard) {
                    grp[0]->launch(grp, st_, chunk_);
                    launches_ += chunk_;
                    e = cudaGetLastError();
                    for (LoopReq *r : grp)
                        if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_sc, r->sc, sizeof(Scal), cudaMemcpyDeviceToHost, st_);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
                    bool all_done = true;
                    for (LoopReq *r : grp) all_done = all_done && r->h_sc->done;
                    if (all_done) break;
                }
                for (LoopReq *r : grp) {
                    if (e == cudaSuccess) e = cudaEventRecord(r->finished, st_);
                    r->err = e;
                }
            }
        }
    }

    int device_;
    int chunk_;
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
