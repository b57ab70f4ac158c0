// C ABI of the FFT phase-field-fracture RVE library (sm_103a): argument checks, error mapping
// and dispatch to the engine of the configured precision (pff_engine.cuh).
#include <thread>

#include "pff_engine.cuh"

using namespace pffeng;

// ================================================================================================
// C ABI
// ================================================================================================
struct rve_s {
    rve_config cfg;
    std::unique_ptr<EngineBase> e;
};

#define GUARD_BEGIN try {
#define GUARD_END                                                                    \
    }                                                                                \
    catch (const CudaError &ce) {                                                    \
        g_last_error = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);       \
        return RVE_ECUDA;                                                            \
    }                                                                                \
    catch (const StatusError &se) {                                                  \
        g_last_error = se.msg;                                                       \
        return se.code;                                                              \
    }                                                                                \
    catch (...) {                                                                    \
        g_last_error = "unknown error";                                              \
        return RVE_ECUDA;                                                            \
    }

extern "C" {

void rve_config_default(rve_config *c) {
    std::memset(c, 0, sizeof(*c));
    c->dim = 2;
    c->n[0] = 64; c->n[1] = 64; c->n[2] = 1;
    c->ell = 2.0;
    c->k_res = 1e-6;
    c->split = RVE_SPLIT_NONE;
    c->precision = RVE_FP64;
    c->history = 1;
    c->f[1] = 1.0;
    c->tol_mech = 1e-12;
    c->tol_dmg = 1e-12;
    c->tol_root = 1e-13;
    c->tol_stag = 1e-10;
    c->max_mech_iters = 20000;
    c->max_dmg_iters = 20000;
    c->max_root_evals = 200;
    c->max_stag_iters = 300;
    c->anderson_m = 5;
    c->fracture_ratio = 0.01;
    c->stream = nullptr;
    c->solver = RVE_SOLVER_STAGGERED;
}

static bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

int rve_config_validate(const rve_config *cfg) {
    if (!cfg) return RVE_EINVAL;
    if (cfg->dim != 2 && cfg->dim != 3) return RVE_EINVAL;
    if (!pow2_in(cfg->n[0], 4, 1024) || !pow2_in(cfg->n[1], 4, 1024)) return RVE_EINVAL;
    if (cfg->dim == 2 && cfg->n[2] != 1) return RVE_EINVAL;
    if (cfg->dim == 3 && cfg->n[2] != 1 && !pow2_in(cfg->n[2], 4, 1024)) return RVE_EINVAL;
    if ((long long)cfg->n[0] * cfg->n[1] * cfg->n[2] > (1LL << 24)) return RVE_EINVAL;
    {
        // the x passes reduce with full-warp shuffles: their CTAs need at least one whole warp
        const int TL = cfg->n[0] / 4;
        const long long pairs = (long long)cfg->n[1] * cfg->n[2] / 2;
        const long long RP = std::min<long long>(std::max(1, 128 / TL), pairs);
        if (RP * TL < 32) {
            g_last_error = "grid too small: the x passes need (nx/4) * min(128/(nx/4), ny*nz/2) >= 32";
            return RVE_EINVAL;
        }
    }
    if (!(cfg->ell > 0) || cfg->k_res < 0 || cfg->anderson_m < 0 || cfg->anderson_m > 5) return RVE_EINVAL;
    if (cfg->split != RVE_SPLIT_NONE && cfg->split != RVE_SPLIT_SPECTRAL) return RVE_EINVAL;
    if (cfg->split == RVE_SPLIT_SPECTRAL && cfg->dim != 2) return RVE_EINVAL;  // split: plane strain only
    if (cfg->solver != RVE_SOLVER_STAGGERED && cfg->solver != RVE_SOLVER_NEWTON) return RVE_EINVAL;
    if (cfg->solver == RVE_SOLVER_NEWTON && cfg->split != RVE_SPLIT_NONE) return RVE_EINVAL;  // not linearised
    if (cfg->solver == RVE_SOLVER_NEWTON && cfg->precision != RVE_FP64) {
        // BiCGSTAB on the coupled single-precision system broke down before its tolerance
        g_last_error = "the Newton solver runs in FP64 only";
        return RVE_EINVAL;
    }
    if (cfg->precision != RVE_FP64 && cfg->precision != RVE_FP32R) return RVE_EINVAL;
    return RVE_OK;
}

int rve_create(const rve_config *cfg, rve_handle *out) {
    if (!cfg || !out) return RVE_EINVAL;
    *out = nullptr;
    if (int rc = rve_config_validate(cfg)) return rc;
    GUARD_BEGIN
    auto *h = new rve_s();
    h->cfg = *cfg;
    try {
        if (cfg->precision == RVE_FP64) h->e.reset(make_engine_f64(*cfg));
        else h->e.reset(make_engine_f32(*cfg));
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    return RVE_OK;
    GUARD_END
}

int set_microstructure(rve_handle h, const rve_micro *m) {
    if (!h || !m) return RVE_EINVAL;
    GUARD_BEGIN
    h->e->crack_len_ = m->crack_kind == RVE_CRACK_NONE ? 0 : m->crack_len;
    return h->e->set_micro(m);
    GUARD_END
}

int step_dissipation(rve_handle h, double dtau, rve_step_result *out) {
    if (!h) return RVE_EINVAL;
    GUARD_BEGIN
    return h->e->step(dtau, out);
    GUARD_END
}

// One increment of each handle, the solves run in lockstep (pff_batch.cuh): a host thread per
// handle runs that handle's own control; the iteration loops of the equilibrium and damage solves
// of all handles are launched together, one kernel launch per pass for every handle of the batch.
static int step_one_guarded(rve_handle h, double dtau, rve_step_result *out) {
    GUARD_BEGIN
    return h->e->step(dtau, out);
    GUARD_END
}

// ---- lockstep batching (pff_batch.cuh) -----------------------------------------------------------
struct rve_batch_group_s {
    Batcher bat;
    // groups serve threads that step independently (the request server): a batch also leaves
    // once its first loop has waited 200 us, so no one stalls on another's host work
    rve_batch_group_s(int dev) : bat(dev, 8, 200.0) {}
};

// One increment of a handle whose thread has joined the group: the solve loops go through the
// group's Batcher; the thread leaves the group when the increment is done.
static int step_joined(rve_handle h, Batcher *bat, double dtau, rve_step_result *out) {
    int rc;
    try {
        h->e->batcher = bat;
        rc = step_one_guarded(h, dtau, out);
    } catch (...) {
        rc = RVE_ECUDA;
    }
    h->e->batcher = nullptr;
    bat->leave();
    return rc;
}

int rve_batch_group_create(rve_batch_group *out) {
    if (!out) return RVE_EINVAL;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RVE_ECUDA;
    auto *g = new rve_batch_group_s(dev);
    if (g->bat.status() != cudaSuccess) {
        delete g;
        return RVE_ECUDA;
    }
    *out = g;
    return RVE_OK;
}

int rve_batch_group_destroy(rve_batch_group g) {
    if (!g) return RVE_EINVAL;
    delete g;
    return RVE_OK;
}

int rve_step_in_group(rve_handle h, rve_batch_group g, double dtau, rve_step_result *out) {
    if (!h || !g) return RVE_EINVAL;
    if (h->e->cfg.split != RVE_SPLIT_NONE || h->e->cfg.solver != RVE_SOLVER_STAGGERED || h->e->timing)
        return RVE_EINVAL;
    g->bat.join();
    return step_joined(h, &g->bat, dtau, out);
}

int rve_step_batch(rve_handle *hs, int n, const double *dtau, rve_step_result *out) {
    if (!hs || !dtau || n < 1 || n > 256) return RVE_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !(dtau[i] > 0.0)) return RVE_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return RVE_EINVAL;
        EngineBase *a = hs[0]->e.get(), *b = hs[i]->e.get();
        if (!b->micro_set) return RVE_ESTATE;
        const rve_config &ca = a->cfg, &cb = b->cfg;
        if (cb.dim != ca.dim || cb.n[0] != ca.n[0] || cb.n[1] != ca.n[1] || cb.n[2] != ca.n[2] ||
            cb.precision != ca.precision || cb.split != RVE_SPLIT_NONE || ca.split != RVE_SPLIT_NONE ||
            cb.solver != RVE_SOLVER_STAGGERED || ca.solver != RVE_SOLVER_STAGGERED || b->cw_y != a->cw_y ||
            b->cw_z != a->cw_z || b->g.Px != a->g.Px || b->timing || a->timing) {
            g_last_error = "rve_step_batch: the handles must share grid, precision and column tiles, use the "
                           "staggered solver without the split, and have timing off";
            return RVE_EINVAL;
        }
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RVE_ECUDA;
    std::vector<int> rc(n, RVE_OK);
    {
        Batcher bat(dev);
        if (bat.status() != cudaSuccess) return RVE_ECUDA;
        // every participant joins before any thread starts, so that the first loops already batch
        for (int i = 0; i < n; ++i) bat.join();
        std::vector<std::thread> th;
        for (int i = 0; i < n; ++i) {
            th.emplace_back([&, i] {
                cudaSetDevice(dev);
                rve_step_result r{};
                rc[i] = step_joined(hs[i], &bat, dtau[i], &r);
                if (out) out[i] = r;
            });
        }
        for (auto &t : th) t.join();
    }
    for (int i = 0; i < n; ++i)
        if (rc[i] != RVE_OK) return rc[i];
    return RVE_OK;
}

int effective_toughness(rve_handle h, double *g_eff) {
    if (!h || !g_eff) return RVE_EINVAL;
    if (!h->e->micro_set) return RVE_ESTATE;
    if (!h->e->S.fractured) return RVE_ENOTFRACTURED;
    *g_eff = h->e->toughness_value();
    return RVE_OK;
}

int effective_toughness_functional(rve_handle h, double *g_eff) {
    if (!h || !g_eff) return RVE_EINVAL;
    if (!h->e->micro_set) return RVE_ESTATE;
    if (!h->e->S.fractured) return RVE_ENOTFRACTURED;
    *g_eff = h->e->toughness_functional_value();
    return RVE_OK;
}

int rve_get_field(rve_handle h, int field, double *host, size_t n) {
    if (!h || !host) return RVE_EINVAL;
    GUARD_BEGIN
    return h->e->get_field(field, host, n);
    GUARD_END
}

int rve_set_field(rve_handle h, int field, const double *host, size_t n) {
    if (!h || !host) return RVE_EINVAL;
    GUARD_BEGIN
    return h->e->set_field(field, host, n);
    GUARD_END
}

int rve_get_scalars(rve_handle h, rve_scalars *s) {
    if (!h || !s) return RVE_EINVAL;
    *s = h->e->S;
    return RVE_OK;
}

int rve_set_scalars(rve_handle h, const rve_scalars *s) {
    if (!h || !s) return RVE_EINVAL;
    h->e->S = *s;
    return RVE_OK;
}

int rve_mech_solve(rve_handle h, int *iters) {
    if (!h) return RVE_EINVAL;
    if (!h->e->micro_set) return RVE_ESTATE;
    GUARD_BEGIN
    int it = 0;
    int rc = h->e->mech_solve_committed(it);
    if (iters) *iters = it;
    return rc;
    GUARD_END
}

int rve_damage_solve(rve_handle h, double E, double *Dv, int *iters) {
    if (!h) return RVE_EINVAL;
    if (!h->e->micro_set) return RVE_ESTATE;
    GUARD_BEGIN
    int it = 0;
    double d = 0.0;
    int rc = h->e->damage_eval_api(E, d, it);
    if (Dv) *Dv = d;
    if (iters) *iters = it;
    return rc;
    GUARD_END
}

int rve_dissipation(rve_handle h, const double *phi_host, double *Dv, double *Gv) {
    if (!h || !phi_host) return RVE_EINVAL;
    if (!h->e->micro_set) return RVE_ESTATE;
    GUARD_BEGIN
    double d = 0.0, gm = 0.0;
    int rc = h->e->dissipation_host(phi_host, d, gm);
    if (Dv) *Dv = d;
    if (Gv) *Gv = gm;
    return rc;
    GUARD_END
}

// Checkpoint layout: rve_scalars | curve length | curve | raw device buffers (phi, H, psi_ini,
// strain fluctuation in the handle's precision and Mandel layout, committed strain in FP64), so
// a reload continues the load path bit-exactly.
int rve_save(rve_handle h, void *buf, size_t *len) {
    if (!h || !len) return RVE_EINVAL;
    GUARD_BEGIN
    auto *e = h->e.get();
    const size_t need = sizeof(rve_scalars) + sizeof(size_t) + e->curve.size() * sizeof(rve_step_result) + e->state_bytes();
    if (!buf) { *len = need; return RVE_OK; }
    if (*len < need) return RVE_EINVAL;
    char *p = (char *)buf;
    std::memcpy(p, &e->S, sizeof(rve_scalars)); p += sizeof(rve_scalars);
    size_t nc = e->curve.size();
    std::memcpy(p, &nc, sizeof(size_t)); p += sizeof(size_t);
    std::memcpy(p, e->curve.data(), nc * sizeof(rve_step_result)); p += nc * sizeof(rve_step_result);
    e->save_state(p);
    *len = need;
    return RVE_OK;
    GUARD_END
}

int rve_load(rve_handle h, const void *buf, size_t len) {
    if (!h || !buf) return RVE_EINVAL;
    GUARD_BEGIN
    auto *e = h->e.get();
    if (!e->micro_set) return RVE_ESTATE;
    const char *p = (const char *)buf;
    if (len < sizeof(rve_scalars) + sizeof(size_t)) return RVE_EINVAL;
    rve_scalars s;
    std::memcpy(&s, p, sizeof(s)); p += sizeof(s);
    size_t nc;
    std::memcpy(&nc, p, sizeof(size_t)); p += sizeof(size_t);
    const size_t need = sizeof(rve_scalars) + sizeof(size_t) + nc * sizeof(rve_step_result) + e->state_bytes();
    if (len != need) return RVE_EINVAL;
    std::vector<rve_step_result> cv(nc);
    std::memcpy(cv.data(), p, nc * sizeof(rve_step_result)); p += nc * sizeof(rve_step_result);
    e->load_state(p);
    e->S = s;
    e->curve = cv;
    return RVE_OK;
    GUARD_END
}

int rve_timing_enable(rve_handle h, int on) {
    if (!h) return RVE_EINVAL;
    h->e->timing = on != 0;
    h->e->timing_reset();
    return RVE_OK;
}

int rve_timing_get(rve_handle h, int kind, double *total_ms, long *launches, double *bytes_per_launch) {
    return rve_timing_get_flops(h, kind, total_ms, launches, bytes_per_launch, nullptr);
}

int rve_timing_get_flops(rve_handle h, int kind, double *total_ms, long *launches, double *bytes_per_launch,
                         double *flops_per_launch) {
    if (!h || kind < 0 || kind > 9) return RVE_EINVAL;
    GUARD_BEGIN
    double ms = 0.0, b = 0.0, f = 0.0;
    long n = 0;
    h->e->timing_get(kind, ms, n, b, f);
    if (total_ms) *total_ms = ms;
    if (launches) *launches = n;
    if (bytes_per_launch) *bytes_per_launch = b;
    if (flops_per_launch) *flops_per_launch = f;
    return RVE_OK;
    GUARD_END
}

long rve_launch_count(rve_handle h) { return h ? h->e->launches : 0; }

int rve_tile_config(rve_handle h, int *cw_y, int *cw_z) {
    if (!h || !cw_y || !cw_z) return RVE_EINVAL;
    *cw_y = h->e->cw_y;
    *cw_z = h->e->g.nz >= 4 ? h->e->cw_z : 0;
    return RVE_OK;
}

int rve_destroy(rve_handle h) {
    if (!h) return RVE_EINVAL;
    delete h;
    return RVE_OK;
}

const char *rve_strerror(int s) {
    switch (s) {
    case RVE_OK: return "ok";
    case RVE_EINVAL: return "invalid argument";
    case RVE_ENOMEM: return "device allocation failed";
    case RVE_ESTATE: return "call out of order";
    case RVE_ENOCONV: return g_last_error.empty() ? "iteration did not converge" : g_last_error.c_str();
    case RVE_ENOROOT: return g_last_error.empty() ? "dissipation constraint could not be bracketed" : g_last_error.c_str();
    case RVE_ETIMEOUT: return "device wait timed out";
    case RVE_ENOTFRACTURED: return "fracture point not reached";
    case RVE_ECUDA: return g_last_error.empty() ? "CUDA error" : g_last_error.c_str();
    case RVE_EBREAKDOWN: return g_last_error.empty() ? "CG breakdown or non-finite value" : g_last_error.c_str();
    default: return "unknown status";
    }
}

}  // extern "C"
