// Request server for many RVE toughness solves on one GPU (continuous batching).
//
// Each request is one RVE (configuration + microstructure, copied at submission) solved by
// repeated dissipation increments until the fracture point or an increment cap. Worker threads
// run admitted requests concurrently, each on its own handle and CUDA stream, so the kernels of
// different RVEs overlap on the device. Requests of one size class (grid and precision) step
// through a shared lockstep group (rve_step_in_group): the solve loops of the requests of a class
// that are in flight at the same moment run as one batched launch per pass, and requests join and
// leave their class's group as they are admitted and retired. Admission is first-come first-served
// under two limits: the number of workers (slots) and an HBM budget checked against each request's
// device footprint (rve_footprint_bytes). A request that fails is retired with its status; the
// others keep running. Results are collected with rve_server_wait.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <thread>
#include <vector>

#include "../../include/pff_rve.h"

namespace pffserve {

struct Request {
    long id;
    rve_config cfg;
    int n_inc;
    double dtau;
    size_t bytes;
    double t_submit;
    // owned copies of the microstructure
    std::vector<int32_t> gid;
    std::vector<double> Cc, R, Gc, cn, beta;
    rve_micro m;
};

struct Server {
    int max_inflight;
    size_t budget;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::unique_ptr<Request>> queue;
    std::vector<rve_request_result> done;
    std::vector<std::thread> workers;
    size_t reserved = 0, peak_bytes = 0;
    int inflight = 0, peak_inflight = 0;
    long submitted = 0, finished = 0;
    bool stop = false;
    int device = 0;
    // off by default: requests stepping concurrently, each on its own stream with graph-launched
    // solve loops, measured faster than lockstep batches of plain launches on every grid class
    bool batching = false;
    // one lockstep group per size class: (dim, nx, ny, nz, precision)
    std::map<std::tuple<int, int, int, int, int>, rve_batch_group> groups;
    rve_batch_group group_for(const rve_config &c) {
        if (!batching || c.split != RVE_SPLIT_NONE || c.solver != RVE_SOLVER_STAGGERED) return nullptr;
        std::lock_guard<std::mutex> lk(mu);
        auto key = std::make_tuple(c.dim, c.n[0], c.n[1], c.n[2], c.precision);
        auto it = groups.find(key);
        if (it != groups.end()) return it->second;
        rve_batch_group g = nullptr;
        if (rve_batch_group_create(&g) != RVE_OK) return nullptr;
        groups[key] = g;
        return g;
    }
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    void run_one(Request &q, rve_request_result &r) {
        r.id = q.id;
        r.status = RVE_OK;
        r.toughness = NAN;
        rve_handle h = nullptr;
        int rc = rve_create(&q.cfg, &h);
        if (rc) { r.status = rc; return; }
        rc = set_microstructure(h, &q.m);
        if (!rc) {
            const long nvox = (long)q.cfg.n[0] * q.cfg.n[1] * q.cfg.n[2];
            rve_batch_group grp = group_for(q.cfg);
            for (int i = 0; i < q.n_inc; ++i) {
                rve_step_result s;
                rc = grp ? rve_step_in_group(h, grp, q.dtau, &s) : step_dissipation(h, q.dtau, &s);
                if (rc) break;
                r.n_done = s.n;
                r.E_last = s.E;
                r.Sigma_last = s.Sigma;
                r.T_last = s.T;
                r.Sigma_max = std::max(r.Sigma_max, s.Sigma);
                r.voxel_updates += (long)(s.mech_iters + s.dmg_iters) * nvox;
                if (s.fractured) {
                    r.fractured = 1;
                    break;
                }
            }
            if (!rc && r.fractured) rc = effective_toughness(h, &r.toughness);
        }
        r.status = rc;
        rve_destroy(h);
    }

    void worker() {
        cudaSetDevice(device);
        for (;;) {
            std::unique_ptr<Request> q;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] {
                    return stop || (!queue.empty() && (inflight == 0 || reserved + queue.front()->bytes <= budget));
                });
                if (stop && queue.empty()) return;
                if (queue.empty()) continue;
                q = std::move(queue.front());
                queue.pop_front();
                reserved += q->bytes;
                ++inflight;
                peak_inflight = std::max(peak_inflight, inflight);
                peak_bytes = std::max(peak_bytes, reserved);
            }
            rve_request_result r;
            std::memset(&r, 0, sizeof(r));
            r.t_submit = q->t_submit;
            r.t_start = now();
            run_one(*q, r);
            r.t_end = now();
            {
                std::lock_guard<std::mutex> lk(mu);
                reserved -= q->bytes;
                --inflight;
                ++finished;
                done.push_back(r);
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
    }
};

}  // namespace pffserve

using namespace pffserve;

struct rve_server_s {
    Server s;
};

extern "C" {

size_t rve_footprint_bytes(const rve_config *c) {
    if (!c) return 0;
    const size_t N = (size_t)c->n[0] * c->n[1] * (c->dim == 3 ? c->n[2] : 1);
    const size_t w = c->precision == RVE_FP32R ? 4 : 8;
    const size_t NS = c->dim == 2 ? 3 : 6;
    const size_t m = (size_t)std::max(0, std::min(5, c->anderson_m));
    size_t b = N * (2 * 4 + 8 * w + 8)          // grain ids, scalar fields, crack source
             + N * NS * (4 * w + 2 * 8)         // equilibrium CG vectors, strain tracking
             + N * (4 * w)                      // damage CG vectors
             + N * 2 * (m + 1) * 8              // Anderson history
             + N * 6 * 8                        // host transfer staging
             + N * NS * 2 * w * 2;              // half spectra (padded)
    if (c->split == RVE_SPLIT_SPECTRAL) b += N * 3 * w;
    if (c->solver == RVE_SOLVER_NEWTON) b += N * (NS + 1) * 11 * w;  // Newton iterate and BiCGSTAB vectors
    return b + (size_t)(24 * 65536) * 8 + (4u << 20);  // reduction partials, tables, slack
}

int rve_server_create(int max_inflight, size_t hbm_budget_bytes, rve_server *out) {
    if (!out || max_inflight < 1 || max_inflight > 256) return RVE_EINVAL;
    auto *sv = new rve_server_s();
    sv->s.max_inflight = max_inflight;
    sv->s.budget = hbm_budget_bytes;
    cudaGetDevice(&sv->s.device);
    for (int i = 0; i < max_inflight; ++i) sv->s.workers.emplace_back([sv] { sv->s.worker(); });
    *out = sv;
    return RVE_OK;
}

int rve_server_submit(rve_server sv, long id, const rve_config *cfg, const rve_micro *m, int n_inc, double dtau) {
    if (!sv || !cfg || !m || !m->grain_id || !m->C_cubic || !m->R || !m->Gc || n_inc < 1 || !(dtau > 0))
        return RVE_EINVAL;
    // the grid fixes how many grain ids are copied below: check it (as rve_create will) first
    if (int rc = rve_config_validate(cfg)) return rc;
    if (m->n_grains <= 0) return RVE_EINVAL;
    auto q = std::make_unique<Request>();
    q->id = id;
    q->cfg = *cfg;
    q->cfg.stream = nullptr;  // every request gets its own stream
    q->n_inc = n_inc;
    q->dtau = dtau;
    q->bytes = rve_footprint_bytes(cfg);
    const size_t N = (size_t)cfg->n[0] * cfg->n[1] * (cfg->dim == 3 ? cfg->n[2] : 1);
    const int G = m->n_grains;
    q->gid.assign(m->grain_id, m->grain_id + N);
    q->Cc.assign(m->C_cubic, m->C_cubic + 3 * G);
    q->R.assign(m->R, m->R + 9 * G);
    q->Gc.assign(m->Gc, m->Gc + G);
    if (m->cleave_n) q->cn.assign(m->cleave_n, m->cleave_n + 3 * G);
    if (m->beta) q->beta.assign(m->beta, m->beta + G);
    q->m = *m;
    q->m.grain_id = q->gid.data();
    q->m.C_cubic = q->Cc.data();
    q->m.R = q->R.data();
    q->m.Gc = q->Gc.data();
    q->m.cleave_n = m->cleave_n ? q->cn.data() : nullptr;
    q->m.beta = m->beta ? q->beta.data() : nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->s.mu);
        q->t_submit = sv->s.now();
        sv->s.queue.push_back(std::move(q));
        ++sv->s.submitted;
    }
    sv->s.cv_work.notify_all();
    return RVE_OK;
}

int rve_server_wait(rve_server sv, rve_request_result *out, int max, double timeout_s, int *n_out) {
    if (!sv || !n_out || (max > 0 && !out)) return RVE_EINVAL;
    std::unique_lock<std::mutex> lk(sv->s.mu);
    auto ready = [&] { return !sv->s.done.empty() || sv->s.finished == sv->s.submitted; };
    if (timeout_s > 0) sv->s.cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    int n = std::min<int>(max, (int)sv->s.done.size());
    for (int i = 0; i < n; ++i) out[i] = sv->s.done[i];
    sv->s.done.erase(sv->s.done.begin(), sv->s.done.begin() + n);
    *n_out = n;
    return RVE_OK;
}

int rve_server_stats(rve_server sv, int *peak_inflight, size_t *peak_bytes, long *pending) {
    if (!sv) return RVE_EINVAL;
    std::lock_guard<std::mutex> lk(sv->s.mu);
    if (peak_inflight) *peak_inflight = sv->s.peak_inflight;
    if (peak_bytes) *peak_bytes = sv->s.peak_bytes;
    if (pending) *pending = sv->s.submitted - sv->s.finished;
    return RVE_OK;
}

int rve_server_set_batching(rve_server sv, int on) {
    if (!sv) return RVE_EINVAL;
    std::lock_guard<std::mutex> lk(sv->s.mu);
    sv->s.batching = on != 0;
    return RVE_OK;
}

int rve_server_destroy(rve_server sv) {
    if (!sv) return RVE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->s.mu);
        sv->s.stop = true;
    }
    sv->s.cv_work.notify_all();
    for (auto &t : sv->s.workers) t.join();
    for (auto &kv : sv->s.groups) rve_batch_group_destroy(kv.second);
    delete sv;
    return RVE_OK;
}

}  // extern "C"
