// Engine and C ABI of the FFT phase-field-fracture RVE library (sm_103a).
//
// One handle = one periodic voxel RVE resident on the device. An increment (Sec. 4.1) is the
// staggered fixed point of Eq. (SystemDisany):
//   1. equilibrium at unit load, Fourier-Galerkin CG (Eq. (GFourier)) on the strain fluctuation;
//   2. the load factor E >= 0 with D(phi(E)) = tau^n (Eq. (SystemDisanyc)); each evaluation is an
//      FFT-preconditioned CG solve of (Gc/l + 2 H_E) phi - div(Gc l A grad phi) = 2 H_E
//      (Eqs. (SystemDisanyb), (gamFunct), (HistoryNumIni));
//   3. Anderson mixing of the staggered map phi -> phi(E) (the accelerated staggering of Storvik
//      et al., cited in Sec. 4.1), stopped by the three ratios of Eq. (errors_crack).
// The monolithic Newton-Raphson increment of Sec. 4.1 (BiCGSTAB on the coupled Jacobian,
// pff_newton.cuh) is the alternative solver of the same equations (rve_config.solver).
// Every field operation runs in the kernels of pff_kernels.cuh / pff_functors.cuh /
// pff_newton.cuh; the host keeps only scalar control: the search on E (secant predictor,
// bracket, secant/Illinois steps), the m x m Anderson least-squares problem, the BiCGSTAB
// scalars and the stopping tests.
#pragma once

#include <cuda_runtime.h>
#include <sys/stat.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pff_rve.h"
#include "pff_batch.cuh"
#include "pff_common.cuh"
#include "pff_functors.cuh"
#include "pff_kernels.cuh"
#include "pff_newton.cuh"

using namespace pff;

namespace pffeng {

struct CudaError {
    cudaError_t e;
    const char *what;
};
struct StatusError {
    int code;
    std::string msg;
};

#define CK(call)                                                         \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) throw CudaError{e_, #call};               \
    } while (0)

inline thread_local std::string g_last_error;

// NVTX range for profilers (nsys, ncu --nvtx): increments, solves and control evaluations show as
// named ranges on the host timeline. Without an attached tool the calls return at once.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// ------------------------------------------------------------------------------------------------
// Setup kernels
// ------------------------------------------------------------------------------------------------

// Per-grain tables. Grains [0, G) are the material grains, [G, 2G) their crack-voxel copies with
// stiffness x crack_mult. Rotated cubic stiffness (Eq. (Crot)) in closed form:
//   C^r_ijkl = C12 d_ij d_kl + C44 (d_ik d_jl + d_il d_jk) + (C11 - C12 - 2 C44) sum_m R_im R_jm R_km R_lm,
// the isotropic part being rotation invariant. Cleavage tensor A = I + beta (I - n n), n the rotated
// weak-plane normal, projected on the plane in 2D (Eq. (PFFani)).
template <typename T>
__global__ void k_build_tables(int G, int dim, const double *Cc, const double *R, const double *Gc,
                               const double *cn, const double *beta, double ell, double crack_mult, T *Cm,
                               T *acoef, T *Ktab, T *GcTab, T *Atab, T *acoefC, T *KtabC, T *lam, T *mu) {
    int gg = blockIdx.x * blockDim.x + threadIdx.x;
    if (gg >= 2 * G) return;
    const int g0 = gg % G;
    const double mult = gg >= G ? crack_mult : 1.0;
    const double c11 = Cc[3 * g0], c12 = Cc[3 * g0 + 1], c44 = Cc[3 * g0 + 2];
    const double dl = c11 - c12 - 2.0 * c44;
    const double *Rg = R + 9 * g0;
    const int NS = dim == 2 ? 3 : 6;
    const int ii3[6] = {0, 1, 2, 1, 0, 0}, jj3[6] = {0, 1, 2, 2, 2, 1};
    const int ii2[3] = {0, 1, 0}, jj2[3] = {0, 1, 1};
    const double sq2 = 1.41421356237309504880;
    auto Cr = [&](int i, int j, int k, int l) {
        double v = c12 * (i == j) * (k == l) + c44 * ((i == k) * (j == l) + (i == l) * (j == k));
        for (int m = 0; m < 3; ++m) v += dl * Rg[3 * i + m] * Rg[3 * j + m] * Rg[3 * k + m] * Rg[3 * l + m];
        return v;
    };
    for (int a = 0; a < NS; ++a) {
        const int i = dim == 2 ? ii2[a] : ii3[a], j = dim == 2 ? jj2[a] : jj3[a];
        const double wa = (i == j) ? 1.0 : sq2;
        for (int b = 0; b < NS; ++b) {
            const int k = dim == 2 ? ii2[b] : ii3[b], l = dim == 2 ? jj2[b] : jj3[b];
            const double wb = (k == l) ? 1.0 : sq2;
            Cm[(size_t)gg * NS * NS + a * NS + b] = (T)(mult * wa * wb * Cr(i, j, k, l));
        }
    }
    // cleavage tensor
    double n[3] = {1.0, 0.0, 0.0};
    const double *nl = cn ? cn + 3 * g0 : n;
    double nr[3];
    for (int i = 0; i < 3; ++i) nr[i] = Rg[3 * i] * nl[0] + Rg[3 * i + 1] * nl[1] + Rg[3 * i + 2] * nl[2];
    const double be = beta ? beta[g0] : 0.0;
    double A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = (i == j) + be * ((i == j) - nr[i] * nr[j]);
    double As[6];
    if (dim == 2) { As[0] = A[0][0]; As[1] = A[1][1]; As[2] = A[0][1]; As[3] = As[4] = As[5] = 0.0; }
    else { As[0] = A[0][0]; As[1] = A[1][1]; As[2] = A[2][2]; As[3] = A[1][2]; As[4] = A[0][2]; As[5] = A[0][1]; }
    const double gc = Gc[g0];
    for (int s = 0; s < 6; ++s) {
        Atab[(size_t)gg * 6 + s] = (T)As[s];
        Ktab[(size_t)gg * 6 + s] = (T)(gc * ell * As[s]);
        KtabC[(size_t)gg * 6 + s] = (T)(ell * ell * As[s]);
    }
    acoef[gg] = (T)(gc / ell);
    acoefC[gg] = (T)1.0;
    GcTab[gg] = (T)gc;
    lam[gg] = (T)(mult * c12);
    mu[gg] = (T)(mult * c44);
}

static __global__ void k_crack_setup(long long N, int nx, int ny, const int *gid0, int G, int kind, int row, int x0,
                              int len, int *gid, double *phi_disc) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int x = (int)(v % nx);
    const int y = (int)((v / nx) % ny);
    int g = gid0[v];
    double pd = 0.0;
    if (kind != RVE_CRACK_NONE && len > 0 && y == row) {
        const int rel = ((x - x0) % nx + nx) % nx;
        if (rel < len) {
            g += G;
            if (kind == RVE_CRACK_CPFE) pd = 1.0;
            else if (rel == 0 || rel == len - 1) pd = 1.0;
        }
    }
    gid[v] = g;
    phi_disc[v] = pd;
}

// Loop condition of a solve captured as a conditional (while) graph node: keep iterating while
// the device scalars say the solve is not done. The solve always ends: the update kernels set
// done at convergence, at the iteration cap, on breakdown and on a non-finite scalar.
static __global__ void k_loop_cond(cudaGraphConditionalHandle h, const Scal *sc) {
    cudaGraphSetConditional(h, sc->done ? 0u : 1u);
}

static __global__ void k_init_scal(Scal *sc, double tol2, int max_iters, double abar, double bbar, double eta2) {
    sc->done = 0; sc->flag = 0; sc->iters = 0; sc->first = 1; sc->max_iters = max_iters;
    sc->tol2 = tol2; sc->beta = 0.0; sc->alpha = 0.0; sc->counter = 0u; sc->abar = abar; sc->bbar = bbar;
    sc->eta2 = eta2;
}

// The correction d of one refinement pass, projected onto compatible strains and added to the
// FP64 solution: x += P[d], d = 0. The FP32 CG leaves rounding-level parts in d that are not
// compatible; those whose stress is divergence-free are invisible to the equilibrium residual
// P[g C : (f + x)], so without the projection they would accumulate in x (and in the stress)
// while the FP64 residual converges. P (the symmetric-strain Galerkin projection) is the
// orthogonal projection onto compatible, mean-free strain fields.
template <typename T, int NS>
struct ProCorrection {  // d, the field to project
    static constexpr int NR = 0;
    static constexpr int RW = NS;
    bool skip_if_done;
    const T *d;
    long long N;
    __device__ void eval(long long v, T *out, double *) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) out[a] = ldro(d + a * N + v);
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};
template <typename T, int NS>
struct EpiAddCorrection {  // x += P[d] (FP64), d = 0
    static constexpr int NR = 0;
    static constexpr int RW = 3 * NS;  // x read + written (double), d written
    bool skip_if_done;
    double *x;
    T *d;
    long long N;
    __device__ void apply(long long v, const T *val, double *) const {
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const size_t i = (size_t)a * N + v;
            x[i] += (double)val[a];
            d[i] = (T)0;
        }
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// ---- pointwise functors used by the engine ------------------------------------------------------
template <typename T>
struct PwSetupMeans {  // mean acoef, mean trace(Ktab)/d, mean trace(KtabC)/d
    static constexpr int NR = 3;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const int *gid;
    const T *acoef, *Ktab, *KtabC;
    int dim;
    __device__ void apply(long long v, double *acc) const {
        const int g = gid[v];
        acc[0] += (double)acoef[g];
        const T *K = Ktab + (size_t)g * 6, *Kc = KtabC + (size_t)g * 6;
        double tk = (double)K[0] + (double)K[1] + (dim == 3 ? (double)K[2] : 0.0);
        double tc = (double)Kc[0] + (double)Kc[1] + (dim == 3 ? (double)Kc[2] : 0.0);
        acc[1] += tk / dim;
        acc[2] += tc / dim;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->red[0] = t[0]; sc->red[1] = t[1]; sc->red[2] = t[2]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

template <typename T>
struct PwMax {
    static constexpr int NR = 1;
    static constexpr bool MAXRED = true;
    bool skip_if_done;
    const T *f;
    __device__ void apply(long long v, double *acc) const { acc[0] = fmax(acc[0], (double)f[v]); }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->red[0] = t[0]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

template <typename T>
struct PwScaleCopy {  // out = s * in
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *in;
    T *out;
    double s;
    __device__ void apply(long long v, double *) const { out[v] = (T)(s * (double)in[v]); }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

template <typename T>
struct PwPsiIni {  // psi_ini = max(0, -gamma'/g'(phi)) = max(0, gamma' / (2 (1 - phi)))  (Eq. (Enini))
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *gp, *phi;
    T *psi_ini, *H;
    __device__ void apply(long long v, double *) const {
        const double val = (double)gp[v] / (2.0 * (1.0 - (double)phi[v]));
        const T r = (T)(val > 0.0 ? val : 0.0);
        psi_ini[v] = r;
        H[v] = r;
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Staggered error on the strain, eps = E (f + x) against the previous iterate (tracking copy),
// in the degraded energy norm |d|^2 = sum d : g(phi) C : d (Mandel: d . g Cm d).
template <typename T, int NS>
struct PwStagEps {
    static constexpr int NR = 2;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *x, *Cm, *phi;
    const int *gid;
    double *eps_it;
    double f[NS];
    double E, k;
    long long N;
    __device__ void apply(long long v, double *acc) const {
        double e[NS], d[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            const size_t i = a * N + v;
            e[a] = E * (f[a] + (double)x[i]);
            d[a] = e[a] - eps_it[i];
            eps_it[i] = e[a];
        }
        const T *C = Cm + (size_t)gid[v] * NS * NS;
        const double ph = (double)phi[v];
        const double gp = (1.0 - ph) * (1.0 - ph) + k;
        double ed = 0.0, ee = 0.0;
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            double sd = 0.0, se = 0.0;
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                sd += (double)C[a * NS + b] * d[b];
                se += (double)C[a * NS + b] * e[b];
            }
            ed += d[a] * sd;
            ee += e[a] * se;
        }
        acc[0] += gp * ed;
        acc[1] += gp * ee;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->red[0] = t[0]; sc->red[1] = t[1]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

template <typename T>
struct PwStagPhi {
    static constexpr int NR = 2;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *pn, *p;
    __device__ void apply(long long v, double *acc) const {
        const double a = (double)pn[v], d = a - (double)p[v];
        acc[0] += d * d;
        acc[1] += a * a;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->red[2] = t[0]; sc->red[3] = t[1]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// Committed macroscopic stress Sigma = <sigma> : f and E_mec = sum g(phi) E^2 psi1.
template <typename T, int NS>
struct PwCommit {
    static constexpr int NR = 2;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *Cm, *x, *phi, *psi1;
    const int *gid;
    double f[NS];
    double E, k;
    long long N;
    __device__ void apply(long long v, double *acc) const {
        const T *C = Cm + (size_t)gid[v] * NS * NS;
        double u[NS];
#pragma unroll
        for (int a = 0; a < NS; ++a) u[a] = f[a] + (double)x[a * N + v];
        const double ph = (double)phi[v];
        const double gp = (1.0 - ph) * (1.0 - ph) + k;
        double sf = 0.0;
#pragma unroll
        for (int a = 0; a < NS; ++a) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < NS; ++b) s += (double)C[a * NS + b] * u[b];
            sf += s * f[a];
        }
        acc[0] += gp * E * sf;
        acc[1] += gp * E * E * (double)psi1[v];
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->red[4] = t[0]; sc->red[5] = t[1]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

// Start of the next solve of a control search: with (x_b, d_b) the last solution and its kept
// divergence and (x_a, d_a) the one before, x_b <- x_b + w (x_b - x_a) (secant extrapolation in E,
// w = 0: none), likewise d_b, and (x_a, d_a) <- the old (x_b, d_b).
template <typename T>
struct PwSecantStart {
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    T *xb, *xa, *db, *da;
    T w;
    __device__ void apply(long long v, double *) const {
        const T pb = xb[v], pa = xa[v], qb = db[v], qa = da[v];
        xa[v] = pb;
        da[v] = qb;
        if (w != (T)0) {
            xb[v] = pb + w * (pb - pa);
            db[v] = qb + w * (qb - qa);
        }
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Anderson: Gram matrix of the residual differences dF_a = R_{a+1} - R_a (R_j = G_j - X_j) and
// their products with the newest residual, K <= 5 columns.
struct AAPtrs {
    const double *X[6];
    const double *G[6];
};

template <typename T>
struct PwAAGram {
    static constexpr int NR = 20;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    AAPtrs h;
    int K;  // number of differences (history length - 1)
    __device__ void apply(long long v, double *acc) const {
        // fixed trip counts with guards keep R and dF in registers
        double R[6], RK = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            R[j] = j <= K ? h.G[j][v] - h.X[j][v] : 0.0;
            if (j == K) RK = R[j];
        }
        double dF[5];
#pragma unroll
        for (int a = 0; a < 5; ++a) dF[a] = a < K ? R[a + 1] - R[a] : 0.0;
        int idx = 0;
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int b = a; b < 5; ++b) {
                if (a < K && b < K) acc[idx] += dF[a] * dF[b];
                ++idx;
            }
#pragma unroll
        for (int a = 0; a < 5; ++a)
            if (a < K) acc[15 + a] += dF[a] * RK;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const {
            for (int i = 0; i < 20; ++i) sc->red[i] = t[i];
        }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

template <typename T>
struct PwAAMix {  // phi = G_K - sum_a gamma_a (G_{a+1} - G_a)
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    AAPtrs h;
    int K;
    double gam[5];
    T *out;
    __device__ void apply(long long v, double *) const {
        double r = h.G[K][v];
        for (int a = 0; a < K; ++a) r -= gam[a] * (h.G[a + 1][v] - h.G[a][v]);
        out[v] = (T)r;
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Committed total strain of a Newton increment: eps = E f + e (Mandel, FP64).
struct F6 {
    double f[6];
};
template <typename T>
__global__ void k_nr_total_strain(long long N, int NS, const T *e, double E, F6 f, double *eps) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= N) return;
    for (int a = 0; a < NS; ++a) eps[a * N + v] = E * f.f[a] + (double)e[a * N + v];
}

// Tensor-component conversion (xx, yy, zz, yz, xz, xy) <-> Mandel, and stress evaluation.
template <typename T>
__global__ void k_mandel_to_tensor(long long N, int dim, const T *src, double scale, const double *f, double *dst) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= N) return;
    const double r2 = 0.70710678118654752440;
    if (dim == 2) {
        dst[0 * N + v] = scale * ((f ? f[0] : 0.0) + (double)src[0 * N + v]);
        dst[1 * N + v] = scale * ((f ? f[1] : 0.0) + (double)src[1 * N + v]);
        dst[2 * N + v] = scale * ((f ? f[2] : 0.0) + (double)src[2 * N + v]) * r2;
    } else {
        for (int a = 0; a < 6; ++a)
            dst[a * N + v] = scale * ((f ? f[a] : 0.0) + (double)src[a * N + v]) * (a < 3 ? 1.0 : r2);
    }
}

template <typename T>
__global__ void k_tensor_to_mandel(long long N, int dim, const double *src, T *dst) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= N) return;
    const double s2 = 1.41421356237309504880;
    const int NS = dim == 2 ? 3 : 6;
    for (int a = 0; a < NS; ++a) dst[a * N + v] = (T)(src[a * N + v] * (a < (dim == 2 ? 2 : 3) ? 1.0 : s2));
}

template <typename T>
__global__ void k_stress(long long N, int dim, const T *Cm, const int *gid, const T *phi, double k, const double *eps,
                         double *sig) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int NS = dim == 2 ? 3 : 6;
    const T *C = Cm + (size_t)gid[v] * NS * NS;
    const double ph = (double)phi[v];
    const double gp = (1.0 - ph) * (1.0 - ph) + k;
    for (int a = 0; a < NS; ++a) {
        double s = 0.0;
        for (int b = 0; b < NS; ++b) s += (double)C[a * NS + b] * eps[b * N + v];
        sig[a * N + v] = gp * s;
    }
}

template <typename T>
__global__ void k_copy_cast(long long n, const T *src, double *dst) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v < n) dst[v] = (double)src[v];
}
template <typename T>
__global__ void k_cast_copy(long long n, const double *src, T *dst) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v < n) dst[v] = (T)src[v];
}

// eps_k = f + x (Newton linearisation point of the split equilibrium).
template <typename T>
struct PwEpsK {
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *x;
    T *epsk;
    T f[3];
    long long N;
    __device__ void apply(long long v, double *) const {
        for (int a = 0; a < 3; ++a) epsk[a * N + v] = f[a] + x[a * N + v];
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Inner (Newton) CG stopping test relative to the initial residual.
static __global__ void k_inner_tol(Scal *sc, double eta2) {
    if (!sc->done) { sc->tol2 = eta2; sc->scale2 = sc->rr0; }
}

// psi1 = psi+(f + x): the crack driving energy with the split.
template <typename T>
struct PwPsi1Split {
    static constexpr int NR = 0;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *x, *lam, *mu;
    const int *gid;
    T *psi1;
    T f[3];
    long long N;
    __device__ void apply(long long v, double *) const {
        T e[3], sp[3], sm[3], pp, pm;
        for (int a = 0; a < 3; ++a) e[a] = f[a] + x[a * N + v];
        const int g = gid[v];
        split_sigma(e, lam[g], mu[g], sp, sm, pp, pm);
        psi1[v] = pp;
    }
    struct Fin { __device__ void operator()(const double *) const {} };
    __device__ Fin fin(Scal *) const { return Fin{}; }
};

// Committed Sigma = <sigma(E eps1)> : f = E <g sigma+(eps1) + sigma-(eps1)> : f and
// E_mec = E^2 sum (g psi+(eps1) + psi-(eps1)) (the split is positively homogeneous).
template <typename T>
struct PwCommitSplit {
    static constexpr int NR = 2;
    static constexpr bool MAXRED = false;
    bool skip_if_done;
    const T *x, *phi, *lam, *mu;
    const int *gid;
    double f[3];
    double E, k;
    long long N;
    __device__ void apply(long long v, double *acc) const {
        double e[3], sp[3], sm[3], pp, pm;
        for (int a = 0; a < 3; ++a) e[a] = f[a] + (double)x[a * N + v];
        const int g = gid[v];
        split_sigma(e, (double)lam[g], (double)mu[g], sp, sm, pp, pm);
        const double ph = (double)phi[v];
        const double gp = (1.0 - ph) * (1.0 - ph) + k;
        double sf = 0.0;
        for (int a = 0; a < 3; ++a) sf += (gp * sp[a] + sm[a]) * f[a];
        acc[0] += E * sf;
        acc[1] += E * E * (gp * pp + pm);
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->red[4] = t[0]; sc->red[5] = t[1]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

template <typename T>
__global__ void k_stress_split(long long N, const T *lam, const T *mu, const int *gid, const T *phi, double k,
                               const double *eps, double *sig) {
    long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= N) return;
    double e[3], sp[3], sm[3], pp, pm;
    for (int a = 0; a < 3; ++a) e[a] = eps[a * N + v];
    const int g = gid[v];
    split_sigma(e, (double)lam[g], (double)mu[g], sp, sm, pp, pm);
    const double ph = (double)phi[v];
    const double gp = (1.0 - ph) * (1.0 - ph) + k;
    for (int a = 0; a < 3; ++a) sig[a * N + v] = gp * sp[a] + sm[a];
}

template <typename C> struct OpNone {
    bool skip_if_done;
    __device__ void apply(const Geom &, int, int, int, const C *, C *) const {}
};

// ------------------------------------------------------------------------------------------------
// Small dense helper: pseudo-inverse solve of a symmetric PSD m x m system by cyclic Jacobi.
// ------------------------------------------------------------------------------------------------
inline void pinv_solve(int m, const double *Min, const double *b, double rcond, double *x) {
    double A[5][5], V[5][5];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) { A[i][j] = Min[i * m + j]; V[i][j] = (i == j); }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = i + 1; j < m; ++j) off += A[i][j] * A[i][j];
        if (off < 1e-300) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                if (A[p][q] == 0.0) continue;
                const double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < m; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < m; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    double lmax = 0.0;
    for (int i = 0; i < m; ++i) lmax = std::max(lmax, std::fabs(A[i][i]));
    for (int i = 0; i < m; ++i) x[i] = 0.0;
    for (int k = 0; k < m; ++k) {
        const double lam = A[k][k];
        if (!(std::fabs(lam) > rcond * lmax) || lam == 0.0) continue;
        double c = 0.0;
        for (int i = 0; i < m; ++i) c += V[i][k] * b[i];
        c /= lam;
        for (int i = 0; i < m; ++i) x[i] += c * V[i][k];
    }
}

// ------------------------------------------------------------------------------------------------
// Column-tile table of the autotuner: process-wide, backed by a text cache file of lines
// "<key> <cw_y> <cw_z>" (the last line for a key wins).
// ------------------------------------------------------------------------------------------------
constexpr int kColumnPassRev = 2;  // 16 points per lane on lines of 16-128 points
inline std::mutex g_tile_mu;
inline std::mutex g_tune_mu;  // one measurement at a time, so concurrent handles do not skew it
inline std::map<std::string, std::pair<int, int>> g_tiles;
inline bool g_tiles_loaded = false;

inline std::string tile_cache_path() {
    const char *p = std::getenv("PFF_TILE_CACHE");
    if (p && *p) return p;
    const char *x = std::getenv("XDG_CACHE_HOME");
    std::string base;
    if (x && *x) base = x;
    else {
        const char *h = std::getenv("HOME");
        if (!h || !*h) return std::string();
        base = std::string(h) + "/.cache";
    }
    return base + "/pff_gb300/tiles.txt";
}

inline void tile_load_locked() {
    if (g_tiles_loaded) return;
    g_tiles_loaded = true;
    const std::string path = tile_cache_path();
    if (path.empty()) return;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char key[512];
    int y, z;
    while (std::fscanf(f, "%511s %d %d", key, &y, &z) == 3) g_tiles[key] = {y, z};
    std::fclose(f);
}

inline bool tile_lookup(const std::string &key, int &y, int &z) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    tile_load_locked();
    auto it = g_tiles.find(key);
    if (it == g_tiles.end()) return false;
    y = it->second.first;
    z = it->second.second;
    return true;
}

inline void tile_store(const std::string &key, int y, int z) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    tile_load_locked();
    g_tiles[key] = {y, z};
    const std::string path = tile_cache_path();
    if (path.empty()) return;
    // create the directory chain; on failure the table stays in memory only
    for (size_t i = 1; i < path.size(); ++i)
        if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
    FILE *f = std::fopen(path.c_str(), "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d\n", key.c_str(), y, z);
    std::fclose(f);
}

// The x passes of the equilibrium CG iteration, timed on their own (timing kinds 8, 9).
template <class P> struct is_cg_dir : std::false_type {};
template <typename U, int NSx> struct is_cg_dir<pff::ProCGCG<U, NSx>> : std::true_type {};
template <class P> struct is_cg_epi : std::false_type {};
template <typename U, int NSx> struct is_cg_epi<pff::EpiCGCG<U, NSx>> : std::true_type {};

// ------------------------------------------------------------------------------------------------
// The engine
// ------------------------------------------------------------------------------------------------
struct SetupInfo {
    double amean, bbar, bbar_cte;
};

// Precision-independent part of a handle: configuration, committed scalars, load curve.
struct EngineBase {
    rve_config cfg;
    Geom g;
    int cw_y = 2, cw_z = 2;  // column tile widths of the y and z passes (autotuned)
    int aw = 16;             // warps per CTA of the column passes at most (PFF_AXIS_WARPS)
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int NS = 3, D = 2;
    long long N = 0;
    bool micro_set = false;
    rve_scalars S{};
    std::vector<rve_step_result> curve;
    long launches = 0;
    int crack_len_ = 0;
    bool timing = false;
    Batcher *batcher = nullptr;  // set while the handle steps inside rve_step_batch (lockstep solves)
    virtual ~EngineBase() {}
    virtual int set_micro(const rve_micro *m) = 0;
    virtual int step(double dtau, rve_step_result *out) = 0;
    virtual int get_field(int field, double *host, size_t n) = 0;
    virtual int set_field(int field, const double *host, size_t n) = 0;
    virtual int mech_solve_committed(int &iters) = 0;
    virtual int damage_eval_api(double E, double &Dv, int &iters) = 0;
    virtual int dissipation_host(const double *phi_host, double &Dv, double &Gv) = 0;
    virtual size_t state_bytes() const = 0;
    virtual void save_state(char *p) = 0;
    virtual void load_state(const char *p) = 0;
    virtual void timing_reset() = 0;
    virtual void timing_get(int kind, double &ms, long &n, double &bytes, double &flops) = 0;
    double crack_area() const { return (double)(g.nx - crack_len_) * (D == 3 ? g.nz : 1); }
    double toughness_value() const { return (double)N / crack_area() * (S.T - 0.5 * S.Sigma * S.E); }
    double toughness_functional_value() const { return (S.D - S.tau0) / crack_area(); }
};

template <typename T>
struct Engine : EngineBase {
    typedef typename cplx_of<T>::type C;
    static constexpr bool kSingle = sizeof(T) == 4;
    // device memory
    std::vector<void *> allocs;
    int *gid0 = nullptr, *gid = nullptr;
    T *Cm = nullptr, *acoef = nullptr, *Ktab = nullptr, *GcTab = nullptr, *Atab = nullptr, *acoefC = nullptr,
      *KtabC = nullptr, *lamT = nullptr, *muT = nullptr;
    T *phi = nullptr, *phi_trial = nullptr, *phi_cur = nullptr, *H = nullptr, *Hcur = nullptr, *psi_ini = nullptr,
      *psi1 = nullptr, *tmpf = nullptr;
    double *phi_disc = nullptr;
    T *mx = nullptr, *mr = nullptr, *mp = nullptr, *mq = nullptr;
    T *dr = nullptr, *dz = nullptr, *dp = nullptr, *dq = nullptr;
    double *eps_it = nullptr, *eps_com = nullptr, *xh = nullptr, *gh = nullptr, *dtmp = nullptr;
    C *spec = nullptr;
    std::map<int, C *> tw;
    Scal *sc = nullptr, *sc2 = nullptr, *h_sc = nullptr, *sc3 = nullptr;
    double *partials = nullptr;
    int G = 0;
    bool iso_damage = true;
    SetupInfo si{};
    double fM[6];
    T *xi_x = nullptr, *xi_y = nullptr, *xi_z = nullptr;
    // timing
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    size_t ev_used = 0;
    // per launch: kernel class (1 k_axis, 2 k_x_fwd, 3 k_x_inv, 4 k_x_mid, 5 k_pointwise), mechanics
    // projection pass?, algorithmic bytes and FFT flops
    // sub: 1 = the mechanics projection pass, 2 / 3 = the forward / inverse x pass of the
    // equilibrium CG iteration (single kernels inside kinds 1, 2, 3; reported as kinds 0, 8, 9)
    struct EvMeta { int kind; int sub; double bytes, flops; };
    std::vector<EvMeta> ev_meta;
    double bytes_mech_axis = 0.0;
    std::map<const void *, size_t> smem_set;
    std::set<const void *> carveout_set;
    // CUDA graphs of one iteration chunk, keyed by (solver kind, solution buffer, coefficient
    // pointer): the kernels of a chunk take only pointers and the device scalar block, so one
    // captured graph is replayed for every chunk of every later solve of the same kind.
    cudaStream_t cap_st = nullptr;
    struct GraphEntry { cudaGraphExec_t exec; long nodes; };
    std::map<std::tuple<int, const void *, const void *>, GraphEntry> graphs;
    bool use_graphs = true;

    // Whole iterative solves as one graph launch: a conditional while node whose body is one
    // iteration plus k_loop_cond. Built once per key by capturing `body` into the node's body
    // graph; returns false (caller falls back to chunks) when graphs are off or timing is on.
    struct LoopEntry { cudaGraphExec_t exec; long body_nodes; bool failed; };
    std::map<std::tuple<int, const void *, const void *>, LoopEntry> loops;
    bool use_loops = true;
    template <class F> bool run_loop(int kind, const void *a, const void *b, Scal *s, F &&body) {
        if (!use_graphs || !use_loops || timing) return false;
        auto key = std::make_tuple(kind, a, b);
        auto it = loops.find(key);
        if (it == loops.end()) {
            LoopEntry e{nullptr, 0, false};
            if (!cap_st) CK(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
            cudaGraphConditionalHandle h;
            ok = ok && cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
            cudaGraphNode_t node;
            alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
            std::memset(cpbuf, 0, sizeof(cpbuf));
            cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cpbuf);
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            ok = ok && cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
            if (ok) {
                cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
                cudaStream_t keep = st;
                const long l0 = launches;
                st = cap_st;
                ok = cudaStreamBeginCaptureToGraph(cap_st, bodyg, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    try {
                        body();
                        k_loop_cond<<<1, 1, 0, st>>>(h, s);
                        ++launches;
                    } catch (...) {
                        ok = false;
                    }
                    cudaGraph_t out_g;
                    ok = (cudaStreamEndCapture(cap_st, &out_g) == cudaSuccess) && ok;
                }
                st = keep;
                e.body_nodes = launches - l0;
                launches = l0;
                ok = ok && cudaGraphInstantiate(&e.exec, g, 0) == cudaSuccess;
            }
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();  // a refused construction is not an error of the solve
            e.failed = !ok;
            if (!ok) e.exec = nullptr;
            it = loops.emplace(key, e).first;
        }
        if (it->second.failed) return false;
        CK(cudaGraphLaunch(it->second.exec, st));
        return true;
    }
    void count_loop(int kind, const void *a, const void *b, int iters) {
        auto it = loops.find(std::make_tuple(kind, a, b));
        if (it != loops.end() && !it->second.failed) launches += (long)std::max(1, iters) * it->second.body_nodes;
    }

    // Run `body` (which launches one chunk on `st`) as a replay of a cached CUDA graph; the first
    // call of a key launches plainly and the second captures. Falls back to plain launches while
    // per-kernel timing is on (event records cannot sit inside a replayed graph).
    template <class F> void run_chunk(int kind, const void *a, const void *b, F &&body) {
        if (!use_graphs || timing) { body(); return; }
        auto key = std::make_tuple(kind, a, b);
        auto it = graphs.find(key);
        if (it != graphs.end()) {
            if (it->second.exec) {
                CK(cudaGraphLaunch(it->second.exec, st));
                launches += it->second.nodes;
                return;
            }
            // second use: capture on the private stream, then replay on the handle's stream
            if (!cap_st) CK(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
            cudaStream_t keep = st;
            const long l0 = launches;
            st = cap_st;
            CK(cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal));
            try {
                body();
            } catch (...) {
                cudaGraph_t gtmp;
                cudaStreamEndCapture(cap_st, &gtmp);
                st = keep;
                throw;
            }
            cudaGraph_t graph;
            CK(cudaStreamEndCapture(cap_st, &graph));
            st = keep;
            cudaGraphExec_t exec;
            CK(cudaGraphInstantiate(&exec, graph, 0));
            CK(cudaGraphDestroy(graph));
            it->second.exec = exec;
            it->second.nodes = launches - l0;
            launches = l0;
            CK(cudaGraphLaunch(exec, st));
            launches += it->second.nodes;
            return;
        }
        graphs[key] = GraphEntry{nullptr, 0};
        body();
    }

    template <typename P> P *alloc(size_t n) {
        void *p = nullptr;
        if (cudaMalloc(&p, n * sizeof(P)) != cudaSuccess) throw StatusError{RVE_ENOMEM, "cudaMalloc failed"};
        allocs.push_back(p);
        CK(cudaMemsetAsync(p, 0, n * sizeof(P), st));
        return (P *)p;
    }

    explicit Engine(const rve_config &c) {
        cfg = c;
        if (kSingle) {
            // FP32 field arithmetic. The equilibrium is refined on its FP64 residual with an FP64
            // solution, so its tolerance can go far below the FP32 rounding level; the damage
            // solve, the control root and the staggered test see FP32 fields and keep floors
            // at what those resolve.
            cfg.tol_mech = std::max(cfg.tol_mech, 1e-13);
            cfg.tol_dmg = std::max(cfg.tol_dmg, 1e-7);
            cfg.tol_root = std::max(cfg.tol_root, 1e-7);  // D(phi) of FP32 fields resolves ~1e-7
            cfg.tol_stag = std::max(cfg.tol_stag, 1e-7);
        }
        D = c.dim;
        NS = D == 2 ? 3 : 6;
        g.d = D; g.ns = NS;
        g.nx = c.n[0]; g.ny = c.n[1]; g.nz = D == 2 ? 1 : c.n[2];
        auto lg = [](int n) { int l = 0; while ((1 << l) < n) ++l; return l; };
        g.lx = lg(g.nx); g.ly = lg(g.ny); g.lz = lg(g.nz);
        auto cw_of = [](int L) { int TL = L / 4; return std::max(2, std::min(16, 256 / std::max(TL, 1))); };
        cw_y = cw_of(g.ny);
        cw_z = g.nz > 1 ? cw_of(g.nz) : 2;
        // spectra and the kx table are sized for the widest column tile (16); the tile widths
        // and the pitch Px actually used are settled by tune_tiles() below
        g.Px = ((g.nx / 2 + 1 + 15) / 16) * 16;
        g.N = (long long)g.nx * g.ny * g.nz;
        g.Nh = (long long)g.Px * g.ny * g.nz;
        g.invN = 1.0 / (double)g.N;
        N = g.N;
        if (const char *aws = std::getenv("PFF_AXIS_WARPS")) aw = std::max(1, std::min(16, std::atoi(aws)));
        if (c.stream) st = (cudaStream_t)c.stream;
        else { CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own_stream = true; }
        CK(axis_twiddles_init());  // constant-bank twiddles of the column passes (this device)
        try {
            gid = alloc<int>(N); gid0 = alloc<int>(N);
            phi = alloc<T>(N); phi_trial = alloc<T>(N); phi_cur = alloc<T>(N); H = alloc<T>(N); Hcur = alloc<T>(N);
            psi_ini = alloc<T>(N); psi1 = alloc<T>(N); tmpf = alloc<T>(N); phi_disc = alloc<double>(N);
            mx = alloc<T>(NS * N); mr = alloc<T>(NS * N); mp = alloc<T>(NS * N); mq = alloc<T>(NS * N);
            dr = alloc<T>(N); dz = alloc<T>(N); dp = alloc<T>(N); dq = alloc<T>(N);
            eps_it = alloc<double>(NS * N); eps_com = alloc<double>(NS * N);
            const int m = std::max(0, std::min(5, cfg.anderson_m));
            xh = alloc<double>((size_t)(m + 1) * N); gh = alloc<double>((size_t)(m + 1) * N);
            dtmp = alloc<double>(6 * N);
            spec = alloc<C>((size_t)std::max(NS, D) * g.Nh);
            sc = alloc<Scal>(1); sc2 = alloc<Scal>(1);
            partials = alloc<double>(24 * 65536);
            CK(cudaMallocHost(&h_sc, sizeof(Scal)));
            for (int L : {g.nx, g.ny, g.nz}) {
                if (L < 4 || tw.count(L)) continue;
                std::vector<C> h(L);
                for (int m2 = 0; m2 < L; ++m2) {
                    long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)m2 / (long double)L;
                    h[m2].x = (T)std::cos(a);
                    h[m2].y = (T)std::sin(a);
                }
                C *d = alloc<C>(L);
                CK(cudaMemcpyAsync(d, h.data(), L * sizeof(C), cudaMemcpyHostToDevice, st));
                tw[L] = d;
            }
            // frequency tables xi~ = 2 pi k / n with the Nyquist frequency set to zero
            auto xi_host = [](int n, int len, bool half) {
                std::vector<T> v(len, (T)0);
                const int lim = half ? n / 2 + 1 : n;
                for (int k = 0; k < lim && k < len; ++k) {
                    const int kk = k <= n / 2 ? k : k - n;
                    v[k] = (2 * k == n) ? (T)0
                                        : (T)(2.0L * 3.14159265358979323846264338327950288L * (long double)kk / (long double)n);
                }
                return v;
            };
            auto up = [&](const std::vector<T> &h) {
                T *d = alloc<T>(h.size());
                CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
                return d;
            };
            xi_x = up(xi_host(g.nx, g.Px, true));
            xi_y = up(xi_host(g.ny, g.ny, false));
            xi_z = up(xi_host(g.nz, g.nz, false));
            CK(cudaStreamSynchronize(st));
        } catch (...) {
            release();
            throw;
        }
        // load direction in Mandel form
        const double s2 = 1.41421356237309504880;
        if (D == 2) { fM[0] = c.f[0]; fM[1] = c.f[1]; fM[2] = s2 * c.f[5]; }
        else { fM[0] = c.f[0]; fM[1] = c.f[1]; fM[2] = c.f[2]; fM[3] = s2 * c.f[3]; fM[4] = s2 * c.f[4]; fM[5] = s2 * c.f[5]; }
        try {
            tune_tiles();
        } catch (...) {
            release();
            throw;
        }
        // spectral bytes of one mechanics axis launch: read + write NS complex per spectral point
        bytes_mech_axis = 2.0 * NS * (double)g.Nh * sizeof(C);
    }

    // ---- column-tile autotuner -------------------------------------------------------------------
    // The y (and z) passes take CW adjacent kx columns per CTA: wider tiles read longer contiguous
    // runs of each spectral row, narrower ones give more CTAs. The best width depends on the grid,
    // the dimension and the precision, so it is measured: every admissible (cw_y, cw_z) runs the
    // mechanics projection pass on this handle's buffers, and the fastest is kept, in a process-
    // wide table and in a cache file, keyed by device, grid, dimension and precision. Each column
    // is transformed by the same code whatever its tile, so the choice does not change any result.
    // Environment: PFF_TILE_TUNE=0 keeps the built-in widths; PFF_TILE_CW=<y>,<z> forces widths;
    // PFF_TILE_CACHE=<file> names the cache (default $XDG_CACHE_HOME or ~/.cache, pff_gb300/tiles.txt).
    void set_tiles(int cy, int cz) {
        cw_y = cy;
        cw_z = cz;
        const int cw = std::max(cw_y, g.nz >= 4 ? cw_z : 1);
        g.Px = ((g.nx / 2 + 1 + cw - 1) / cw) * cw;
        g.Nh = (long long)g.Px * g.ny * g.nz;
    }
    std::vector<int> tile_candidates(int L) const {
        std::vector<int> v;
        const int NM = std::max(NS, D);
        for (int cw = 1; cw <= 16; cw *= 2) {
            int th;
            size_t sm;
            axis_shape<C>(L, NM, cw, th, sm);
            if (sm <= 200 * 1024) v.push_back(cw);
        }
        if (v.empty()) v.push_back(1);
        return v;
    }
    float time_tiles(int cy, int cz) {
        set_tiles(cy, cz);
        init_sc(sc, 0.0, 0);
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {
            CK(cudaEventRecord(a, st));
            if (NS == 3) spectral<3, 3>(OpProj<C, 3>{false, xitab()}, sc);
            else spectral<6, 6>(OpProj<C, 6>{false, xitab()}, sc);
            CK(cudaEventRecord(b, st));
            CK(cudaEventSynchronize(b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (rep > 0) best = std::min(best, ms);  // the first run warms up
        }
        CK(cudaEventDestroy(a));
        CK(cudaEventDestroy(b));
        return best;
    }
    std::string tile_key() const {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        cudaDeviceProp pr;
        CK(cudaGetDeviceProperties(&pr, dev));
        char buf[512];
        // kColumnPassRev names the column-pass code the timings were taken on: a cache written by
        // another revision of it is not reused
        std::snprintf(buf, sizeof(buf), "%s|sm%d%d|d%d|%dx%dx%d|%s|r%d", pr.name, pr.major, pr.minor, D, g.nx, g.ny,
                      g.nz, kSingle ? "fp32" : "fp64", kColumnPassRev);
        std::string k(buf);
        for (char &ch : k)
            if (ch == ' ') ch = '_';
        return k;
    }
    void tune_tiles() {
        const std::vector<int> cy = tile_candidates(g.ny);
        const std::vector<int> cz = g.nz >= 4 ? tile_candidates(g.nz) : std::vector<int>{cw_z};
        auto admissible = [&](int y, int z) {
            return std::find(cy.begin(), cy.end(), y) != cy.end() && std::find(cz.begin(), cz.end(), z) != cz.end();
        };
        const char *force = std::getenv("PFF_TILE_CW");
        if (force) {
            int y = 0, z = 0;
            const int got = std::sscanf(force, "%d,%d", &y, &z);
            if (g.nz < 4 && got >= 1) z = cw_z;  // no z pass: only the y width matters
            if (got >= 1 && admissible(y, z)) { set_tiles(y, z); return; }
        }
        const char *tune = std::getenv("PFF_TILE_TUNE");
        if (tune && std::string(tune) == "0") { set_tiles(cw_y, cw_z); return; }
        const std::string key = tile_key();
        int y = 0, z = 0;
        if (tile_lookup(key, y, z) && admissible(y, z)) { set_tiles(y, z); return; }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (tile_lookup(key, y, z) && admissible(y, z)) { set_tiles(y, z); return; }
        float best = 1e30f;
        int by = cw_y, bz = cw_z;
        for (int yy : cy)
            for (int zz : cz) {
                const float ms = time_tiles(yy, zz);
                if (ms < best) { best = ms; by = yy; bz = zz; }
            }
        set_tiles(by, bz);
        tile_store(key, by, bz);
    }

    void release() {
        for (auto &kv : loops)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        loops.clear();
        for (auto &kv : graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        graphs.clear();
        if (cap_st) cudaStreamDestroy(cap_st);
        cap_st = nullptr;
        for (auto &e : ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        ev_pool.clear();
        for (void *p : allocs) cudaFree(p);
        allocs.clear();
        if (h_sc) cudaFreeHost(h_sc);
        h_sc = nullptr;
        if (ev_ready) cudaEventDestroy(ev_ready);
        if (ev_finished) cudaEventDestroy(ev_finished);
        ev_ready = ev_finished = nullptr;
        if (own_stream && st) cudaStreamDestroy(st);
        st = nullptr;
    }
    ~Engine() { release(); }
    XiTab<T> xitab() const { return XiTab<T>{xi_x, xi_y, xi_z}; }

    // ---- launch helpers --------------------------------------------------------------------
    static int fail(int code, const char *what) {
        g_last_error = what;
        return code;
    }
    // forward x pass of the FP32 path: the shared-memory carveout at its maximum, so that shared
    // memory does not cap the resident CTAs below what its register bound allows (L1 caching does
    // not help its streaming prologue)
    template <typename K> void prep_x(K kernel, size_t bytes) {
        prep_smem(kernel, bytes);
        if (sizeof(T) != 4 || carveout_set.count((const void *)kernel)) return;
        // not while the stream is being captured into a graph: the attribute is set at the
        // kernel's first launch outside a capture and applies to every later launch
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(st, &cs));
        if (cs != cudaStreamCaptureStatusNone) return;
        CK(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
        carveout_set.insert((const void *)kernel);
    }
    template <typename K> void prep_smem(K kernel, size_t bytes) {
        const void *key = (const void *)kernel;
        auto it = smem_set.find(key);
        // opt in above 32 KB: static shared memory (reduction scratch) adds to the dynamic size
        if (bytes > 32 * 1024 && (it == smem_set.end() || it->second < bytes)) {
            CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
            smem_set[key] = bytes;
        }
    }
    // Events around one launch while timing is on (returns the end event to record after it).
    cudaEvent_t tbeg(int kind, int sub, double bytes, double flops) {
        if (!timing) return nullptr;
        if (ev_used == ev_pool.size()) {
            cudaEvent_t a, b;
            CK(cudaEventCreate(&a)); CK(cudaEventCreate(&b));
            ev_pool.push_back({a, b});
        }
        if (ev_meta.size() < ev_pool.size()) ev_meta.resize(ev_pool.size());
        ev_meta[ev_used] = EvMeta{kind, sub, bytes, flops};
        CK(cudaEventRecord(ev_pool[ev_used].first, st));
        return ev_pool[ev_used++].second;
    }
    void tend(cudaEvent_t e) { if (e) CK(cudaEventRecord(e, st)); }
    // FFT flops of NC transforms of the x rows (two real rows per complex line of nx points).
    double xflops(int nc) const { return (double)nc * 0.5 * (double)g.ny * g.nz * 5.0 * g.nx * g.lx; }
    // Algorithmic bytes of an x pass: nc_spec half-spectrum components and RW field words per voxel.
    template <typename U = T> double xbytes(int nc_spec, int rw) const {
        return (double)nc_spec * (g.nx / 2 + 1) * (double)g.ny * g.nz * sizeof(typename cplx_of<U>::type) +
               (double)rw * N * sizeof(T);
    }
    // Spectral buffer, twiddles and frequency tables of the transforms in precision U: the
    // engine's own for U = T; for U = double in the FP32 engine, a second set used by the FP64
    // residual passes of the iterative refinement (allocated on first use).
    typedef typename cplx_of<double>::type C64;
    C64 *spec64 = nullptr;
    std::map<int, C64 *> tw64;
    double *xi64_x = nullptr, *xi64_y = nullptr, *xi64_z = nullptr;
    template <typename U> typename cplx_of<U>::type *spec_of() {
        if constexpr (std::is_same<U, T>::value) return spec;
        else return spec64;
    }
    template <typename U> const typename cplx_of<U>::type *tw_of(int L) {
        if constexpr (std::is_same<U, T>::value) return tw[L];
        else return tw64[L];
    }
    XiTab<double> xitab64() const { return XiTab<double>{xi64_x, xi64_y, xi64_z}; }
    void ensure_spectral64() {
        if (spec64) return;
        spec64 = alloc<C64>((size_t)std::max(NS, D) * (size_t)(((g.nx / 2 + 1 + 15) / 16) * 16) * g.ny * g.nz);
        for (int L : {g.nx, g.ny, g.nz}) {
            if (L < 4 || tw64.count(L)) continue;
            std::vector<C64> h(L);
            for (int m2 = 0; m2 < L; ++m2) {
                long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)m2 / (long double)L;
                h[m2].x = (double)std::cos(a);
                h[m2].y = (double)std::sin(a);
            }
            C64 *d = alloc<C64>(L);
            CK(cudaMemcpyAsync(d, h.data(), L * sizeof(C64), cudaMemcpyHostToDevice, st));
            tw64[L] = d;
        }
        auto xi_host = [](int n, int len, bool half) {
            std::vector<double> v(len, 0.0);
            const int lim = half ? n / 2 + 1 : n;
            for (int k = 0; k < lim && k < len; ++k) {
                const int kk = k <= n / 2 ? k : k - n;
                v[k] = (2 * k == n) ? 0.0
                                    : (double)(2.0L * 3.14159265358979323846264338327950288L * (long double)kk / (long double)n);
            }
            return v;
        };
        auto up = [&](const std::vector<double> &h) {
            double *d = alloc<double>(h.size());
            CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
            return d;
        };
        xi64_x = up(xi_host(g.nx, ((g.nx / 2 + 1 + 15) / 16) * 16, true));
        xi64_y = up(xi_host(g.ny, g.ny, false));
        xi64_z = up(xi_host(g.nz, g.nz, false));
    }
    template <typename U = T> void xcfg(int &threads, int &blocks, size_t &smem1) const {
        const int TL = g.nx / 4;
        const long long pairs = (long long)g.ny * g.nz / 2;
        int RP = std::max(1, 128 / TL);
        if (RP > pairs) RP = (int)pairs;
        threads = RP * TL;
        blocks = (int)(pairs / RP);
        smem1 = (size_t)RP * g.nx * sizeof(typename cplx_of<U>::type);
    }
    template <int NC, class Pro, typename U = T> void x_fwd(const Pro &pro, Scal *s) {
        int th, bl; size_t sm; xcfg<U>(th, bl, sm);
        auto k = k_x_fwd<U, NC, Pro>;
        prep_x(k, sm * NC);
        cudaEvent_t e = tbeg(std::is_same<U, T>::value ? 2 : 7, is_cg_dir<Pro>::value ? 2 : 0,
                             xbytes<U>(NC, rw_words<Pro>()), xflops(NC));
        k<<<bl, th, sm * NC, st>>>(g, pro, spec_of<U>(), tw_of<U>(g.nx), partials, s);
        CK(cudaGetLastError());
        tend(e);
        ++launches;
    }
    template <int NC, class Epi, typename U = T> void x_inv(const Epi &epi, Scal *s) {
        int th, bl; size_t sm; xcfg<U>(th, bl, sm);
        auto k = k_x_inv<U, NC, Epi>;
        prep_smem(k, sm * NC);
        cudaEvent_t e = tbeg(std::is_same<U, T>::value ? 3 : 7, is_cg_epi<Epi>::value ? 3 : 0,
                             xbytes<U>(NC, rw_words<Epi>()), xflops(NC));
        k<<<bl, th, sm * NC, st>>>(g, spec_of<U>(), epi, tw_of<U>(g.nx), partials, s);
        CK(cudaGetLastError());
        tend(e);
        ++launches;
    }
    template <int NC, class Mid> void x_mid(const Mid &mid, Scal *s) { x_mid2<NC, NC>(mid, s); }
    template <int NCI, int NCO, class Mid> void x_mid2(const Mid &mid, Scal *s) {
        int th, bl; size_t sm; xcfg(th, bl, sm);
        auto k = k_x_mid<T, NCI, NCO, Mid>;
        prep_smem(k, sm * NCI);
        cudaEvent_t e = tbeg(4, 0, xbytes(NCI + NCO, rw_words<Mid>()), xflops(NCI + NCO));
        k<<<bl, th, sm * NCI, st>>>(g, spec, mid, tw[g.nx], s);
        CK(cudaGetLastError());
        tend(e);
        ++launches;
    }
    template <int NCI, int NCO, int MODE, class Op, typename U = T>
    void axis(int ax, const Op &op, Scal *s, bool timed = false) {
        typedef typename cplx_of<U>::type CU;
        const int L = ax == 1 ? g.ny : g.nz;
        int CW = ax == 1 ? cw_y : cw_z;
        const int NM = NCI > NCO ? NCI : NCO;
        int threads;
        size_t sm;
        axis_shape<CU>(L, NM, CW, threads, sm, aw);
        // FP64 passes of the FP32 engine: halve the tuned width until the tile fits (Px stays a
        // multiple of the narrower width)
        while (sm > 200 * 1024 && CW > 1) {
            CW >>= 1;
            axis_shape<CU>(L, NM, CW, threads, sm, aw);
        }
        dim3 grid(g.Px / CW, ax == 1 ? g.nz : g.ny);
        auto k = axis_kernel<U, NCI, NCO, MODE, Op>(L);
        prep_smem(k, sm);
        // timing: `timed` marks the mechanics projection pass. Bytes: the NCI components read and
        // the components written over the half spectrum (the nx/2 + 1 columns, no tile padding);
        // flops: 5 L log2 L per transformed column and component.
        const int nout = MODE == AX_FWD_OP_INV ? NCO : NCI;
        const int ntr = MODE == AX_FWD_OP_INV ? NCI + NCO : NCI;
        const double cols = (double)(g.nx / 2 + 1) * (ax == 1 ? g.nz : g.ny);
        // the FP64 residual passes of the FP32 engine form their own class (7)
        cudaEvent_t e = tbeg(std::is_same<U, T>::value ? 1 : 7, (timed && std::is_same<U, T>::value) ? 1 : 0,
                             (double)(NCI + nout) * cols * L * sizeof(CU),
                             (double)ntr * cols * 5.0 * L * (ax == 1 ? g.ly : g.lz));
        k<<<grid, threads, sm, st>>>(g, ax, CW, spec_of<U>(), spec_of<U>(), op, tw_of<U>(L), s);
        CK(cudaGetLastError());
        tend(e);
        ++launches;
    }
    // Grid of the pointwise kernels. Those that reduce pay a fixed per-CTA cost (block reduction,
    // fence, atomic ticket), which dominated at one voxel per thread; they run 2 CTAs per SM with
    // a grid-stride loop instead. The others take one voxel per thread up to 1184 CTAs.
    int num_sms = 0;
    template <class F> long long pw_blocks(long long n) {
        if (!num_sms) {
            int dev = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        }
        long long bl = (n + 255) / 256;
        const long long cap = F::NR > 0 ? 2LL * num_sms : 1184;
        return bl > cap ? cap : bl;
    }
    template <class F> void pointwise(const F &f, Scal *s) {
        cudaEvent_t e = tbeg(5, 0, (double)rw_words<F>() * N * sizeof(T), 0.0);
        k_pointwise<F><<<(int)pw_blocks<F>(N), 256, 0, st>>>(N, f, partials, s);
        CK(cudaGetLastError());
        tend(e);
        ++launches;
    }
    // Spectral passes between the x passes: 2D one y pass; 3D y, z (with the operator), y. A 3D
    // grid one voxel thick (nz = 1, the plates of Sec. 5) has xi_z = 0 everywhere and needs no z
    // transform: the operator runs in the y pass, as in 2D, with all NS components.
    template <int NCI, int NCO, class Op, typename U = T> void spectral(const Op &op, Scal *s, bool timed = false) {
        typedef typename cplx_of<U>::type CU;
        if (D == 2 || g.nz == 1) {
            axis<NCI, NCO, AX_FWD_OP_INV, Op, U>(1, op, s, timed);
        } else {
            OpNone<CU> nop{op.skip_if_done};
            axis<NCI, NCI, AX_FWD, OpNone<CU>, U>(1, nop, s, timed);
            axis<NCI, NCO, AX_FWD_OP_INV, Op, U>(2, op, s, timed);
            axis<NCO, NCO, AX_INV, OpNone<CU>, U>(1, nop, s, timed);
        }
    }
    void read_sc(Scal *s) {
        CK(cudaMemcpyAsync(h_sc, s, sizeof(Scal), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    void init_sc(Scal *s, double tol, int maxit, double abar = 0.0, double bbar = 0.0, double eta = 0.0) {
        k_init_scal<<<1, 1, 0, st>>>(s, tol * tol, maxit, abar, bbar, eta * eta);
        ++launches;
    }

    // ---- batched launches (rve_step_batch): one launch per pass for several RVEs of this grid -------
    template <class F>
    static SlotArgs<F> slot_args(const std::vector<Engine *> &es, const std::vector<F> &fs, const std::vector<Scal *> &scs) {
        SlotArgs<F> a;
        for (size_t i = 0; i < es.size(); ++i) {
            a.a[i].f = fs[i];
            a.a[i].spec = es[i]->spec;
            a.a[i].partials = es[i]->partials;
            a.a[i].sc = scs[i];
        }
        return a;
    }
    template <int NC, class Pro>
    void x_fwd_b(const std::vector<Engine *> &es, const std::vector<Pro> &fs, const std::vector<Scal *> &scs,
                 cudaStream_t s) {
        int th, bl; size_t sm; xcfg(th, bl, sm);
        auto k = k_x_fwd_b<T, NC, Pro>;
        prep_x(k, sm * NC);
        k<<<dim3(bl, 1, (unsigned)es.size()), th, sm * NC, s>>>(g, slot_args(es, fs, scs), tw[g.nx]);
    }
    template <int NC, class Epi>
    void x_inv_b(const std::vector<Engine *> &es, const std::vector<Epi> &fs, const std::vector<Scal *> &scs,
                 cudaStream_t s) {
        int th, bl; size_t sm; xcfg(th, bl, sm);
        auto k = k_x_inv_b<T, NC, Epi>;
        prep_smem(k, sm * NC);
        k<<<dim3(bl, 1, (unsigned)es.size()), th, sm * NC, s>>>(g, slot_args(es, fs, scs), tw[g.nx]);
    }
    template <int NCI, int NCO, class Mid>
    void x_mid_b(const std::vector<Engine *> &es, const std::vector<Mid> &fs, const std::vector<Scal *> &scs,
                 cudaStream_t s) {
        int th, bl; size_t sm; xcfg(th, bl, sm);
        auto k = k_x_mid_b<T, NCI, NCO, Mid>;
        prep_smem(k, sm * NCI);
        k<<<dim3(bl, 1, (unsigned)es.size()), th, sm * NCI, s>>>(g, slot_args(es, fs, scs), tw[g.nx]);
    }
    template <int NCI, int NCO, int MODE, class Op>
    void axis_b(int ax, const std::vector<Engine *> &es, const std::vector<Op> &fs, const std::vector<Scal *> &scs,
                cudaStream_t s) {
        const int L = ax == 1 ? g.ny : g.nz;
        const int CW = ax == 1 ? cw_y : cw_z;
        const int NM = NCI > NCO ? NCI : NCO;
        int threads;
        size_t sm;
        axis_shape<C>(L, NM, CW, threads, sm, aw);
        auto k = axis_kernel_b<T, NCI, NCO, MODE, Op>(L);
        prep_smem(k, sm);
        k<<<dim3(g.Px / CW, ax == 1 ? g.nz : g.ny, (unsigned)es.size()), threads, sm, s>>>(g, ax, CW,
                                                                                         slot_args(es, fs, scs), tw[L]);
    }
    template <int NCI, int NCO, class Op>
    int spectral_b(const std::vector<Engine *> &es, const std::vector<Op> &fs, const std::vector<Scal *> &scs,
                   cudaStream_t s) {
        if (D == 2 || g.nz == 1) {
            axis_b<NCI, NCO, AX_FWD_OP_INV, Op>(1, es, fs, scs, s);
            return 1;
        }
        std::vector<OpNone<C>> nops(es.size(), OpNone<C>{true});
        axis_b<NCI, NCI, AX_FWD, OpNone<C>>(1, es, nops, scs, s);
        axis_b<NCI, NCO, AX_FWD_OP_INV, Op>(2, es, fs, scs, s);
        axis_b<NCO, NCO, AX_INV, OpNone<C>>(1, es, nops, scs, s);
        return 3;
    }
    // One iteration loop of a solve handed to the Batcher: the equilibrium CG (ProCGCG -> projection
    // -> EpiCGCG) or the damage PCG (ProPCGCG -> preconditioner + gradient -> flux -> divergence ->
    // EpiPCGCG), each RVE with its own functors.
    cudaEvent_t ev_ready = nullptr, ev_finished = nullptr;
    template <class Q> void batch_request(Q &q) {
        if (!ev_ready) {
            CK(cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ev_finished, cudaEventDisableTiming));
        }
        q.e = this;
        q.sc = sc;
        q.h_sc = h_sc;
        q.slot_stream = st;
        q.ready = ev_ready;
        q.finished = ev_finished;
        q.launch_counter = &launches;
        q.launch = &Q::run_iters;
        batcher->run(&q);
        if (q.err != cudaSuccess) throw CudaError{q.err, "batched solve"};
    }
    template <int NSx> struct MechLoop : LoopReq {
        Engine *e = nullptr;
        ProCGCG<T, NSx> dir;
        OpProj<C, NSx> proj;
        EpiCGCG<T, NSx> eq;
        static void run_iters(std::vector<LoopReq *> &grp, cudaStream_t s, int iters) {
            const size_t n = grp.size();
            std::vector<Engine *> es(n);
            std::vector<ProCGCG<T, NSx>> ds(n);
            std::vector<OpProj<C, NSx>> ps(n);
            std::vector<EpiCGCG<T, NSx>> qs(n);
            std::vector<Scal *> scs(n);
            for (size_t i = 0; i < n; ++i) {
                auto *r = static_cast<MechLoop *>(grp[i]);
                es[i] = r->e; ds[i] = r->dir; ps[i] = r->proj; qs[i] = r->eq; scs[i] = r->sc;
            }
            Engine *e0 = es[0];
            long k = 0;
            for (int it = 0; it < iters; ++it) {
                e0->template x_fwd_b<NSx>(es, ds, scs, s);
                k += e0->template spectral_b<NSx, NSx>(es, ps, scs, s);
                e0->template x_inv_b<NSx>(es, qs, scs, s);
                k += 2;
            }
            *grp[0]->launch_counter += k;
        }
    };
    template <int Dx> struct DmgLoop : LoopReq {
        Engine *e = nullptr;
        ProPCGCG<T> pdir;
        OpPrecGrad<C, Dx> pgrad;
        MidFluxU<T, Dx> fluxu;
        OpDiv<C, Dx> divo;
        EpiPCGCG<T> ew;
        static void run_iters(std::vector<LoopReq *> &grp, cudaStream_t s, int iters) {
            const size_t n = grp.size();
            std::vector<Engine *> es(n);
            std::vector<ProPCGCG<T>> a(n);
            std::vector<OpPrecGrad<C, Dx>> b(n);
            std::vector<MidFluxU<T, Dx>> c(n);
            std::vector<OpDiv<C, Dx>> d(n);
            std::vector<EpiPCGCG<T>> w(n);
            std::vector<Scal *> scs(n);
            for (size_t i = 0; i < n; ++i) {
                auto *r = static_cast<DmgLoop *>(grp[i]);
                es[i] = r->e; a[i] = r->pdir; b[i] = r->pgrad; c[i] = r->fluxu; d[i] = r->divo; w[i] = r->ew;
                scs[i] = r->sc;
            }
            Engine *e0 = es[0];
            long k = 0;
            for (int it = 0; it < iters; ++it) {
                e0->template x_fwd_b<1>(es, a, scs, s);
                k += e0->template spectral_b<1, Dx + 1>(es, b, scs, s);
                e0->template x_mid_b<Dx + 1, Dx>(es, c, scs, s);
                k += e0->template spectral_b<Dx, 1>(es, d, scs, s);
                e0->template x_inv_b<1>(es, w, scs, s);
                k += 3;
            }
            *grp[0]->launch_counter += k;
        }
    };

    // ---- mechanics (a1-a5) ---------------------------------------------------------------------
    // ---- FP32 path: mixed-precision iterative refinement of the equilibrium ---------------------
    // x (the unit-load fluctuation) is kept in FP64 (mx64). Each pass evaluates the true residual
    // r = -P[g C : (f + x)] with FP64 transforms and tables, then runs the FP32 single-reduction
    // CG on the correction A d = r (d in md) until <r, r> drops by eta^2 or meets the tolerance,
    // and adds the compatible part P[d] of d to x in FP64 (EpiAddCorrection says why). The solve
    // ends at the first pass whose FP64 residual meets the tolerance. mx then holds x rounded to
    // FP32 for the consumers of the fluctuation.
    double *mx64 = nullptr, *Cm64 = nullptr;
    T *md = nullptr;
    bool mx64_ok = false;
    // inner reduction of each refinement pass; PFF_REFINE_ETA overrides it (tuning)
    double refine_eta = std::getenv("PFF_REFINE_ETA") ? std::atof(std::getenv("PFF_REFINE_ETA")) : 1e-4;
    void ensure_mx64() {
        if (!mx64) mx64 = alloc<double>((size_t)NS * N);
        if (!mx64_ok) {
            k_copy_cast<T><<<(int)((NS * N + 255) / 256), 256, 0, st>>>(NS * N, mx, mx64);
            CK(cudaGetLastError());
            ++launches;
            mx64_ok = true;
        }
    }
    template <int NSx> int mech_solve_refined(const T *phi_in, int &iters) {
        ensure_spectral64();
        ensure_mx64();
        if (!md) md = alloc<T>((size_t)NS * N);
        if (!mw) mw = alloc<T>((size_t)NS * N);
        CK(cudaMemsetAsync(md, 0, sizeof(T) * NS * N, st));
        MechBase<T, NSx> mb{Cm, gid, phi_in, (T)cfg.k_res, N, true};
        ProStressTotal64<NSx> pro64{true, Cm64, gid, (const float *)phi_in, cfg.k_res, mx64, {}, N};
        for (int a = 0; a < NSx; ++a) pro64.f[a] = fM[a];
        OpProj<C64, NSx> proj64{true, xitab64()};
        OpProj<C, NSx> proj{true, xitab()};
        ProCGCG<T, NSx> dir;
        (MechBase<T, NSx> &)dir = mb;
        dir.x = md; dir.r = mr; dir.p = mp; dir.s = mq; dir.w = mw; dir.scr = sc;
        EpiCGCG<T, NSx> eq{true, mw, mr, N};
        const int chunk = timing ? 1 : 8;
        iters = 0;
        bool converged = false;
        for (int pass = 0; pass < 16 && !converged; ++pass) {
            init_sc(sc, cfg.tol_mech, std::max(1, cfg.max_mech_iters - iters), 0.0, 0.0, refine_eta);
            x_fwd<NSx, ProStressTotal64<NSx>, double>(pro64, sc);
            spectral<NSx, NSx, OpProj<C64, NSx>, double>(proj64, sc, true);
            x_inv<NSx, EpiMechInit64<NSx>, double>(EpiMechInit64<NSx>{true, (float *)mr, N}, sc);
            auto iter_body = [&] {
                x_fwd<NSx>(dir, sc);
                spectral<NSx, NSx>(proj, sc, true);
                x_inv<NSx>(eq, sc);
            };
            if (batcher) {
                MechLoop<NSx> q;
                q.dir = dir; q.proj = proj; q.eq = eq;
                batch_request(q);
            } else if (run_loop(1, phi_in, nullptr, sc, iter_body)) {
                read_sc(sc);
                count_loop(1, phi_in, nullptr, h_sc->iters);
            } else {
                for (;;) {
                    run_chunk(1, phi_in, nullptr, [&] {
                        for (int c = 0; c < chunk; ++c) iter_body();
                    });
                    read_sc(sc);
                    if (h_sc->done) break;
                }
            }
            iters += h_sc->iters;
            if (h_sc->flag & FLAG_NONFINITE) return fail(RVE_EBREAKDOWN, "equilibrium CG: non-finite scalar");
            if (h_sc->flag) {
                // FP32 CG breakdown (<p, A p> <= 0 from rounding in a nearly singular system):
                // on a residual already at the rounding floor (within 100 x the tolerance, FP64-
                // verified at the start of this pass) the verified x is kept; otherwise the
                // correction gathered before the breakdown is added and the next pass restarts
                // from the FP64 residual (the pass cap bounds this)
                if (h_sc->rr0 <= 1e4 * h_sc->tol2 * h_sc->scale2) {
                    CK(cudaMemsetAsync(md, 0, sizeof(T) * NS * N, st));
                    converged = true;
                    break;
                }
            } else {
                if (h_sc->iters == 0) { converged = true; break; }  // the FP64 residual met the tolerance
                if (!(h_sc->rr <= h_sc->tol2 * h_sc->scale2) && !(h_sc->rr <= h_sc->eta2 * h_sc->rr0))
                    return fail(RVE_ENOCONV, "equilibrium CG: iteration cap");
            }
            x_fwd<NSx>(ProCorrection<T, NSx>{false, md, N}, sc2);
            spectral<NSx, NSx>(OpProj<C, NSx>{false, xitab()}, sc2);
            x_inv<NSx>(EpiAddCorrection<T, NSx>{false, mx64, md, N}, sc2);
        }
        if (!converged) return fail(RVE_ENOCONV, "equilibrium: iterative refinement did not reach the tolerance");
        k_cast_copy<T><<<(int)((NS * N + 255) / 256), 256, 0, st>>>(NS * N, mx64, mx);
        CK(cudaGetLastError());
        ++launches;
        PwPsi1<T, NSx> ps{false, Cm, mx, gid, psi1, {}, N};
        for (int a = 0; a < NSx; ++a) ps.f[a] = (T)fM[a];
        pointwise(ps, sc);
        return RVE_OK;
    }

    template <int NSx> int mech_solve_t(const T *phi_in, int &iters) {
        if constexpr (kSingle) return mech_solve_refined<NSx>(phi_in, iters);
        MechBase<T, NSx> mb{Cm, gid, phi_in, (T)cfg.k_res, N, true};
        ProStressTotal<T, NSx> pro;
        (MechBase<T, NSx> &)pro = mb;
        pro.x = mx;
        for (int a = 0; a < NSx; ++a) pro.f[a] = (T)fM[a];
        init_sc(sc, cfg.tol_mech, cfg.max_mech_iters);
        OpProj<C, NSx> proj{true, xitab()};
        x_fwd<NSx>(pro, sc);
        spectral<NSx, NSx>(proj, sc, true);
        x_inv<NSx>(EpiMechInit<T, NSx>{true, mr, N}, sc);
        if (!mw) mw = alloc<T>((size_t)NS * N);
        ProCGCG<T, NSx> dir;
        (MechBase<T, NSx> &)dir = mb;
        dir.x = mx; dir.r = mr; dir.p = mp; dir.s = mq; dir.w = mw; dir.scr = sc;
        EpiCGCG<T, NSx> eq{true, mw, mr, N};
        // FP64: one CG pass (as the oracle). FP32: iterative refinement -- each pass restarts CG
        // from the equilibrium residual recomputed from the current strain, until that true
        // residual meets the tolerance (a pass that needs no iteration).
        const int passes = kSingle ? 8 : 1;
        const int chunk = timing ? 1 : 8;  // timed runs launch no iteration past convergence
        iters = 0;
        for (int pass = 0; pass < passes; ++pass) {
            if (pass > 0) {
                init_sc(sc, cfg.tol_mech, std::max(1, cfg.max_mech_iters - iters));
                x_fwd<NSx>(pro, sc);
                spectral<NSx, NSx>(proj, sc, true);
                x_inv<NSx>(EpiMechInit<T, NSx>{true, mr, N}, sc);
            }
            auto iter_body = [&] {
                x_fwd<NSx>(dir, sc);
                spectral<NSx, NSx>(proj, sc, true);
                x_inv<NSx>(eq, sc);
            };
            if (batcher) {
                MechLoop<NSx> q;
                q.dir = dir; q.proj = proj; q.eq = eq;
                batch_request(q);
            } else if (run_loop(1, phi_in, nullptr, sc, iter_body)) {
                read_sc(sc);
                count_loop(1, phi_in, nullptr, h_sc->iters);
            } else {
                for (;;) {
                    run_chunk(1, phi_in, nullptr, [&] {
                        for (int c = 0; c < chunk; ++c) iter_body();
                    });
                    read_sc(sc);
                    if (h_sc->done) break;
                }
            }
            iters += h_sc->iters;
            if (h_sc->flag) return fail(RVE_EBREAKDOWN, "equilibrium CG: breakdown or non-finite scalar");
            if (!(h_sc->rr <= h_sc->tol2 * h_sc->scale2)) return fail(RVE_ENOCONV, "equilibrium CG: iteration cap");
            if (!kSingle || h_sc->iters == 0) break;
        }
        PwPsi1<T, NSx> ps{false, Cm, mx, gid, psi1, {}, N};
        for (int a = 0; a < NSx; ++a) ps.f[a] = (T)fM[a];
        pointwise(ps, sc);
        return RVE_OK;
    }
    int mech_solve(const T *phi_in, int &iters) {
        Range nvtx("equilibrium solve");
        if (cfg.split == RVE_SPLIT_SPECTRAL) return mech_solve_split(phi_in, iters);
        return NS == 3 ? mech_solve_t<3>(phi_in, iters) : mech_solve_t<6>(phi_in, iters);
    }

    // Equilibrium with the spectral split (2D): Newton on P[sigma(f + x)] = 0, each step a CG on
    // the tangent P[K(eps_k) : dx] = -P[sigma(eps_k)] to 1e-3 of its initial residual; stops when
    // |P[sigma]| <= tol_mech |sigma|. The problem is positively homogeneous of degree one, so the
    // unit-load solution scales with E >= 0.
    T *epsk = nullptr, *mw = nullptr, *dw = nullptr;
    // div(K grad x) of the damage field phi_trial as the last solve of the running control search
    // left it (valid while ddiv_ok): the next solve of the same search starts without transforms
    T *ddiv = nullptr;
    bool ddiv_ok = false;
    // The evaluation before the last one of the running search (phi, div at E_prev): the next
    // solve starts from the secant extrapolation in E of the last two solutions. div(K grad phi)
    // is linear in phi, so the kept divergence extrapolates exactly with it.
    T *phi_prev = nullptr, *ddiv_prev = nullptr;
    bool prev_ok = false;
    double E_last = 0.0, E_prev = 0.0;
    int mech_solve_split(const T *phi_in, int &iters) {
        if (!epsk) epsk = alloc<T>((size_t)3 * N);
        ProSplitStress<T> pst{true, mx, phi_in, lamT, muT, gid, (T)cfg.k_res, {}, N};
        for (int a = 0; a < 3; ++a) pst.f[a] = (T)fM[a];
        OpProj<C, 3> proj{true, xitab()};
        PwEpsK<T> ek{false, mx, epsk, {}, N};
        for (int a = 0; a < 3; ++a) ek.f[a] = (T)fM[a];
        ProSplitDir<T> dir{true, mr, epsk, phi_in, lamT, muT, mp, gid, (T)cfg.k_res, sc, N};
        EpiMechQ<T, 3> eq{true, mq, mp, N};
        PwMechUpdate<T, 3> up{true, mx, mr, mp, mq, sc, N};
        iters = 0;
        for (int newton = 0; newton < 100; ++newton) {
            init_sc(sc, cfg.tol_mech, std::max(1, cfg.max_mech_iters - iters));
            x_fwd<3>(pst, sc);
            spectral<3, 3>(proj, sc, true);
            x_inv<3>(EpiMechInit<T, 3>{true, mr, N}, sc);
            read_sc(sc);
            if (h_sc->flag) return RVE_EBREAKDOWN;
            if (h_sc->done) break;
            pointwise(ek, sc);
            k_inner_tol<<<1, 1, 0, st>>>(sc, 1e-6);
            ++launches;
            auto iter_body = [&] {
                x_fwd<3>(dir, sc);
                spectral<3, 3>(proj, sc, true);
                x_inv<3>(eq, sc);
                pointwise(up, sc);
            };
            if (run_loop(2, phi_in, nullptr, sc, iter_body)) {
                read_sc(sc);
                count_loop(2, phi_in, nullptr, h_sc->iters);
            } else {
                for (;;) {
                    run_chunk(2, phi_in, nullptr, [&] {
                        for (int c = 0; c < 8; ++c) iter_body();
                    });
                    read_sc(sc);
                    if (h_sc->done) break;
                }
            }
            iters += h_sc->iters;
            if (h_sc->flag) return fail(RVE_EBREAKDOWN, "split equilibrium: breakdown or non-finite scalar");
            if (iters >= cfg.max_mech_iters) return fail(RVE_ENOCONV, "split equilibrium: CG iteration cap");
            if (newton == 99) return fail(RVE_ENOCONV, "split equilibrium: Newton did not converge in 100 steps");
        }
        mx64_ok = false;  // the split solve updates mx itself
        PwPsi1Split<T> ps{false, mx, lamT, muT, gid, psi1, {}, N};
        for (int a = 0; a < 3; ++a) ps.f[a] = (T)fM[a];
        pointwise(ps, sc);
        return RVE_OK;
    }

    // ---- damage (a6-a8) ------------------------------------------------------------------------
    // Generic FFT-preconditioned CG for  a v - div(K grad v) = rhs, warm-started from x.
    // Damage (mode 0, 1) or enrichment (mode 2) solve. In damage mode *Dx_out receives D(x) of the
    // solution: in FP32 from the final refinement pass, whose residual evaluation computed it from
    // the converged x (no iteration followed); in FP64 from the residual identity of PwDmgEnergy.
    // It is NaN when neither applies (the caller then evaluates D itself).
    // reuse: (damage mode) ddiv holds div(K grad x) for the current x; the first residual is then
    // one pointwise pass. In damage mode ddiv is left valid for the returned x when *Dx_out is
    // finite.
    template <int Dx> int pcg_t(int mode, double E, const DmgCoef<T> &co, const T *rhs, T rhs_scale, T *x,
                                double tol, int maxit, double amean, double bbar, int &iters,
                                double *Dx_out = nullptr, bool reuse = false) {
        if (Dx_out) *Dx_out = NAN;
        if (!ddiv) ddiv = alloc<T>(N);
        T *keep = mode != 2 ? ddiv : nullptr;
        ProDmgInit<T> pi{true, mode, E, psi1, psi_ini, H, Hcur, rhs, x, amean, bbar, (double)co.hmul, N};
        OpGrad<C, Dx> grad{true, xitab()};
        OpDiv<C, Dx> divo{true, xitab()};
        MidFlux<T, Dx> flux{true, co.Ktab, gid};
        if (!dw) dw = alloc<T>(N);
        ProPCGCG<T> pdir{true, x, dr, dp, dq, dz, dw, sc};
        OpPrecGrad<C, Dx> pgrad{true, sc, xitab()};
        MidFluxU<T, Dx> fluxu{true, co.Ktab, gid, dz};
        EpiPCGCG<T> ew{true, co.acoef, gid, co.hmul, co.H, dz, dr, dw};
        // FP64: one PCG pass; FP32: passes restarted from the true residual (see mech_solve_t).
        const int passes = kSingle ? 8 : 1;
        const int chunk = timing ? 1 : 4;
        iters = 0;
        for (int pass = 0; pass < passes; ++pass) {
            init_sc(sc, tol, std::max(1, maxit - iters));
            // r = rhs - L x (true residual), then the single-reduction iteration
            if (pass == 0 && reuse && mode != 2) {
                pointwise(PwDmgInitKept<T>{false, mode, E, psi1, psi_ini, H, Hcur, co, x, ddiv, dr, amean, bbar, N},
                          sc);
            } else {
                x_fwd<1>(pi, sc);
                spectral<1, Dx>(grad, sc);
                x_mid<Dx>(flux, sc);
                spectral<Dx, 1>(divo, sc);
                x_inv<1>(EpiDmgRes<T>{true, co, x, dr, rhs, rhs_scale, keep}, sc);
            }
            auto iter_body = [&] {
                x_fwd<1>(pdir, sc);
                spectral<1, Dx + 1>(pgrad, sc);
                x_mid2<Dx + 1, Dx>(fluxu, sc);
                spectral<Dx, 1>(divo, sc);
                x_inv<1>(ew, sc);
            };
            if (batcher) {
                DmgLoop<Dx> q;
                q.pdir = pdir; q.pgrad = pgrad; q.fluxu = fluxu; q.divo = divo; q.ew = ew;
                batch_request(q);
            } else if (run_loop(3, x, co.Ktab, sc, iter_body)) {
                read_sc(sc);
                count_loop(3, x, co.Ktab, h_sc->iters);
            } else {
                for (;;) {
                    run_chunk(3, x, co.Ktab, [&] {
                        for (int c = 0; c < chunk; ++c) iter_body();
                    });
                    read_sc(sc);
                    if (h_sc->done) break;
                }
            }
            iters += h_sc->iters;
            if (h_sc->flag) return fail(RVE_EBREAKDOWN, "damage CG: breakdown or non-finite scalar");
            if (!(h_sc->rr <= h_sc->tol2 * h_sc->scale2)) return fail(RVE_ENOCONV, "damage CG: iteration cap");
            if (!kSingle || h_sc->iters == 0) break;
        }
        if (Dx_out && mode != 2) {
            if (kSingle) {
                if (h_sc->iters == 0) *Dx_out = h_sc->D;
            } else {
                init_sc(sc2, 0.0, 0);
                pointwise(PwDmgEnergy<T>{false, co, x, dr, rhs, (double)rhs_scale, keep}, sc2);
                read_sc(sc2);
                *Dx_out = h_sc->D;
            }
        }
        return RVE_OK;
    }
    int pcg(int mode, double E, const DmgCoef<T> &co, const T *rhs, T rhs_scale, T *x, double tol, int maxit,
            double amean, double bbar, int &iters, double *Dx_out = nullptr, bool reuse = false) {
        return D == 2 ? pcg_t<2>(mode, E, co, rhs, rhs_scale, x, tol, maxit, amean, bbar, iters, Dx_out, reuse)
                      : pcg_t<3>(mode, E, co, rhs, rhs_scale, x, tol, maxit, amean, bbar, iters, Dx_out, reuse);
    }
    DmgCoef<T> dmg_coef() const { return DmgCoef<T>{acoef, Ktab, gid, (T)2.0, Hcur}; }

    // D(phi) and Gamma(phi) (a9)
    template <int Dx> void dissipation_t(const T *f, double &Dv, double &Gv) {
        init_sc(sc2, 0.0, 0);
        OpGrad<C, Dx> grad{false, xitab()};
        x_fwd<1>(ProField<T>{false, f}, sc2);
        spectral<1, Dx>(grad, sc2);
        x_inv<Dx>(EpiDiss<T, Dx>{false, f, GcTab, Atab, gid, cfg.ell}, sc2);
        read_sc(sc2);
        Dv = h_sc->D;
        Gv = h_sc->Gamma;
    }
    void dissipation(const T *f, double &Dv, double &Gv) {
        if (D == 2) dissipation_t<2>(f, Dv, Gv); else dissipation_t<3>(f, Dv, Gv);
    }

    // phi(E) into phi_trial (warm start = current phi_trial); returns D(phi(E)).
    int damage_eval(double E, double &Dv, int &iters) {
        Range nvtx("damage solve");
        const int mode = cfg.history ? 0 : 1;
        double Dsol;
        const bool reuse = ddiv_ok;
        if (reuse) {
            if (!phi_prev) { phi_prev = alloc<T>(N); ddiv_prev = alloc<T>(N); }
            double w = 0.0;
            if (prev_ok && E_last != E_prev) {
                w = (E - E_last) / (E_last - E_prev);
                if (!(std::fabs(w) <= 4.0)) w = 0.0;  // far outside the last step: no extrapolation
            }
            pointwise(PwSecantStart<T>{false, phi_trial, phi_prev, ddiv, ddiv_prev, (T)w}, sc2);
            E_prev = E_last;
            prev_ok = true;
        } else {
            prev_ok = false;
        }
        ddiv_ok = false;
        int rc = pcg(mode, E, dmg_coef(), Hcur, (T)2.0, phi_trial, cfg.tol_dmg, cfg.max_dmg_iters, si.amean,
                     si.bbar, iters, &Dsol, reuse);
        if (rc) { prev_ok = false; return rc; }
        ddiv_ok = std::isfinite(Dsol);
        if (ddiv_ok) E_last = E;
        else prev_ok = false;
        if (std::isfinite(Dsol)) {
            Dv = Dsol;
        } else {
            double Gm;
            dissipation(phi_trial, Dv, Gm);
        }
        return RVE_OK;
    }

    // ---- setup (a12) -------------------------------------------------------------------------
    int set_micro(const rve_micro *m) override {
        G = m->n_grains;
        if (G <= 0 || !m->grain_id || !m->C_cubic || !m->R || !m->Gc) return RVE_EINVAL;
        for (long long v = 0; v < N; ++v)
            if (m->grain_id[v] < 0 || m->grain_id[v] >= G) return RVE_EINVAL;
        iso_damage = true;
        if (m->beta)
            for (int i = 0; i < G; ++i) iso_damage = iso_damage && (m->beta[i] == 0.0);
        if (cfg.split == RVE_SPLIT_SPECTRAL) {
            for (int i = 0; i < G; ++i) {
                const double c11 = m->C_cubic[3 * i], c12 = m->C_cubic[3 * i + 1], c44 = m->C_cubic[3 * i + 2];
                if (std::fabs(c44 - 0.5 * (c11 - c12)) > 1e-12 * std::fabs(c11)) return RVE_EINVAL;
            }
        }
        if (m->crack_kind != RVE_CRACK_NONE &&
            (m->crack_row < 0 || m->crack_row >= g.ny || m->crack_len <= 0 || m->crack_len > g.nx || m->crack_phi_M <= 0 ||
             m->crack_phi_M >= 1.0))
            return RVE_EINVAL;
        // per-grain tables
        for (void *p : {(void *)Cm, (void *)acoef, (void *)Ktab, (void *)GcTab, (void *)Atab, (void *)acoefC,
                        (void *)KtabC, (void *)lamT, (void *)muT}) {
            if (p) {
                cudaFree(p);
                allocs.erase(std::remove(allocs.begin(), allocs.end(), p), allocs.end());
            }
        }
        const int G2 = 2 * G;
        Cm = alloc<T>((size_t)G2 * NS * NS); acoef = alloc<T>(G2); Ktab = alloc<T>((size_t)G2 * 6);
        GcTab = alloc<T>(G2); Atab = alloc<T>((size_t)G2 * 6); acoefC = alloc<T>(G2); KtabC = alloc<T>((size_t)G2 * 6);
        lamT = alloc<T>(G2); muT = alloc<T>(G2);
        double *dCc, *dR, *dGc, *dcn = nullptr, *dbe = nullptr;
        CK(cudaMalloc(&dCc, sizeof(double) * 3 * G)); CK(cudaMalloc(&dR, sizeof(double) * 9 * G));
        CK(cudaMalloc(&dGc, sizeof(double) * G));
        CK(cudaMemcpyAsync(dCc, m->C_cubic, sizeof(double) * 3 * G, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dR, m->R, sizeof(double) * 9 * G, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dGc, m->Gc, sizeof(double) * G, cudaMemcpyHostToDevice, st));
        if (m->cleave_n) {
            CK(cudaMalloc(&dcn, sizeof(double) * 3 * G));
            CK(cudaMemcpyAsync(dcn, m->cleave_n, sizeof(double) * 3 * G, cudaMemcpyHostToDevice, st));
        }
        if (m->beta) {
            CK(cudaMalloc(&dbe, sizeof(double) * G));
            CK(cudaMemcpyAsync(dbe, m->beta, sizeof(double) * G, cudaMemcpyHostToDevice, st));
        }
        CK(cudaMemcpyAsync(gid0, m->grain_id, sizeof(int) * N, cudaMemcpyHostToDevice, st));
        k_build_tables<T><<<(G2 + 63) / 64, 64, 0, st>>>(G, D, dCc, dR, dGc, dcn, dbe, cfg.ell, m->crack_stiffness, Cm,
                                                          acoef, Ktab, GcTab, Atab, acoefC, KtabC, lamT, muT);
        ++launches;
        if constexpr (kSingle) {
            // FP64 copy of the stiffness table for the FP64 residual of the refinement (the other
            // FP64 tables are built and dropped)
            if (Cm64) {
                cudaFree(Cm64);
                allocs.erase(std::remove(allocs.begin(), allocs.end(), (void *)Cm64), allocs.end());
            }
            Cm64 = alloc<double>((size_t)G2 * NS * NS);
            double *t64;
            const size_t per = 1 + 6 + 1 + 6 + 1 + 6 + 1 + 1;
            CK(cudaMalloc(&t64, sizeof(double) * per * G2));
            double *q = t64;
            double *a1 = q; q += G2; double *a2 = q; q += 6 * G2; double *a3 = q; q += G2; double *a4 = q; q += 6 * G2;
            double *a5 = q; q += G2; double *a6 = q; q += 6 * G2; double *a7 = q; q += G2; double *a8 = q;
            k_build_tables<double><<<(G2 + 63) / 64, 64, 0, st>>>(G, D, dCc, dR, dGc, dcn, dbe, cfg.ell,
                                                                   m->crack_stiffness, Cm64, a1, a2, a3, a4, a5, a6,
                                                                   a7, a8);
            CK(cudaGetLastError());
            ++launches;
            CK(cudaStreamSynchronize(st));
            CK(cudaFree(t64));
        }
        const int cx0 = ((m->crack_x0 % g.nx) + g.nx) % g.nx;
        k_crack_setup<<<(int)((N + 255) / 256), 256, 0, st>>>(N, g.nx, g.ny, gid0, G, m->crack_kind, m->crack_row, cx0,
                                                              m->crack_len, gid, phi_disc);
        ++launches;
        init_sc(sc2, 0, 0);
        pointwise(PwSetupMeans<T>{false, gid, acoef, Ktab, KtabC, D}, sc2);
        read_sc(sc2);
        si.amean = h_sc->red[0] / (double)N;
        si.bbar = h_sc->red[1] / (double)N;
        si.bbar_cte = h_sc->red[2] / (double)N;
        CK(cudaFree(dCc)); CK(cudaFree(dR)); CK(cudaFree(dGc));
        if (dcn) CK(cudaFree(dcn));
        if (dbe) CK(cudaFree(dbe));
        // enriched initial crack
        CK(cudaMemsetAsync(mx, 0, sizeof(T) * NS * N, st));
        mx64_ok = false;
        CK(cudaMemsetAsync(eps_com, 0, sizeof(double) * NS * N, st));
        CK(cudaMemsetAsync(psi1, 0, sizeof(T) * N, st));
        double tau0 = 0.0, Gamma0 = 0.0;
        if (m->crack_kind == RVE_CRACK_NONE) {
            CK(cudaMemsetAsync(phi, 0, sizeof(T) * N, st));
            CK(cudaMemsetAsync(psi_ini, 0, sizeof(T) * N, st));
            CK(cudaMemsetAsync(H, 0, sizeof(T) * N, st));
        } else {
            int rc = cte_init(m->crack_phi_M, tau0, Gamma0);
            if (rc) return rc;
        }
        CK(cudaMemcpyAsync(phi_trial, phi, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(Hcur, H, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
        S = rve_scalars{};
        S.tau = tau0;
        S.tau0 = tau0;
        S.D = tau0;
        S.Gamma = Gamma0;
        curve.clear();
        micro_set = true;
        root_slope = 0.0;
        return RVE_OK;
    }

    // phi_o - l^2 div(A grad phi_o) = phi_disc (Eqs. (damini), (daminiAni), read with l^2),
    // phi_ini = phi_M phi_o / max phi_o, psi_ini = max(0, gamma'(phi_ini) / (2 (1 - phi_ini))) (Eq. (Enini)).
    int cte_init(double phi_M, double &tau0, double &Gamma0) {
        T *phi_disc_T = tmpf;
        k_cast_copy<T><<<(int)((N + 255) / 256), 256, 0, st>>>(N, phi_disc, phi_disc_T);
        ++launches;
        if (iso_damage) {
            init_sc(sc2, 0, 0, 1.0, cfg.ell * cfg.ell);
            OpPrec<C> prec{false, sc2, xitab()};
            x_fwd<1>(ProField<T>{false, phi_disc_T}, sc2);
            spectral<1, 1>(prec, sc2);
            x_inv<1>(EpiStore<T>{false, phi}, sc2);
        } else {
            CK(cudaMemsetAsync(phi, 0, sizeof(T) * N, st));
            DmgCoef<T> co{acoefC, KtabC, gid, (T)0.0, Hcur};
            int it = 0;
            int rc = pcg(2, 0.0, co, phi_disc_T, (T)1.0, phi, kSingle ? 1e-6 : 1e-14, 20000, 1.0, si.bbar_cte, it);
            if (rc) return rc;
        }
        init_sc(sc2, 0, 0);
        pointwise(PwMax<T>{false, phi}, sc2);
        read_sc(sc2);
        const double mx_ = h_sc->red[0];
        if (!(mx_ > 0.0)) return RVE_EINVAL;
        pointwise(PwScaleCopy<T>{false, phi, phi, phi_M / mx_}, sc2);
        // gamma'(phi_ini) = Gc/l phi - div(Gc l A grad phi)
        DmgCoef<T> co0{acoef, Ktab, gid, (T)0.0, Hcur};
        if (D == 2) apply_L<2>(co0, phi, tmpf); else apply_L<3>(co0, phi, tmpf);
        pointwise(PwPsiIni<T>{false, tmpf, phi, psi_ini, H}, sc2);
        dissipation(phi, tau0, Gamma0);
        return RVE_OK;
    }
    template <int Dx> void apply_L(const DmgCoef<T> &co, const T *v, T *out) {
        init_sc(sc2, 0, 0);
        OpGrad<C, Dx> grad{false, xitab()};
        OpDiv<C, Dx> divo{false, xitab()};
        x_fwd<1>(ProField<T>{false, v}, sc2);
        spectral<1, Dx>(grad, sc2);
        x_mid<Dx>(MidFlux<T, Dx>{false, co.Ktab, gid}, sc2);
        spectral<Dx, 1>(divo, sc2);
        x_inv<1>(EpiApply<T>{false, co, v, out}, sc2);
    }

    // ---- control: smallest E >= 0 with D(phi(E)) = tau (a10) -----------------------------------
    int arc_length(double tau, double E_guess, double &E_out, double &D_out, rve_step_result &st_) {
        Range nvtx("control search");
        int it = 0, rc;
        ddiv_ok = false;  // phi_trial was just reset to the staggered iterate
        prev_ok = false;
        double Ep = -1.0, fp = 0.0;
        auto evaluate = [&](double E, double &f) -> int {
            double Dv;
            int r = damage_eval(E, Dv, it);
            st_.dmg_iters += it;
            st_.root_evals += 1;
            eval_iters = it;
            if (r) return r;
            f = Dv - tau;
            D_out = Dv;
            // slope memory for the secant predictor, from evaluations far enough apart that the
            // solve tolerance does not dominate the difference quotient
            if (Ep >= 0.0 && std::fabs(E - Ep) > 1e-3 * std::max(E, Ep)) {
                const double sl = (f - fp) / (E - Ep);
                if (std::isfinite(sl) && sl > 0.0) root_slope = sl;
            }
            Ep = E;
            fp = f;
            return RVE_OK;
        };
        if (E_guess <= 0.0) {
            // scale of E from the mean driving energy (same recipe as the oracle)
            init_sc(sc2, 0, 0);
            pointwise(PwSum<T>{false, psi1}, sc2);
            read_sc(sc2);
            const double pm = std::max(h_sc->red[0] / (double)N, 1e-300);
            E_guess = std::sqrt(si.amean * cfg.ell / (cfg.ell * pm)) * 0.05;
        }
        double E0 = E_guess;
        double f0;
        if ((rc = evaluate(E0, f0))) return rc;
        if (std::fabs(f0) <= cfg.tol_root * tau) { E_out = E0; return RVE_OK; }
        double h = 1e-3 * E0, lo, flo, hi, fhi;
        int guard = 0;
        // Secant predictor from the slope dD/dE of the last root solve, aimed 2% past the root so
        // that it usually brackets it in one evaluation. D(phi(E)) is non-decreasing in E, so
        // this only shortens the search; the root is the same (bracketing below and Illinois).
        if (root_slope > 0.0) {
            double E1 = E0 - 1.02 * f0 / root_slope;
            E1 = std::min(std::max(E1, 0.5 * E0), 2.0 * E0);
            double f1;
            if ((rc = evaluate(E1, f1))) return rc;
            if (std::fabs(f1) <= cfg.tol_root * tau) {
                E_out = E1;
                return RVE_OK;
            }
            if ((f0 < 0.0) != (f1 < 0.0)) {
                if (f0 < 0.0) { lo = E0; flo = f0; hi = E1; fhi = f1; }
                else { lo = E1; flo = f1; hi = E0; fhi = f0; }
                return illinois(tau, lo, flo, hi, fhi, evaluate, E_out);
            }
            // same side: continue the bracket search from the closer point
            h = std::max(std::fabs(E1 - E0), 1e-3 * E0);
            E0 = E1;
            f0 = f1;
        }
        if (f0 < 0.0) {
            lo = E0; flo = f0; hi = lo + h;
            if ((rc = evaluate(hi, fhi))) return rc;
            while (fhi <= 0.0) {
                if (++guard > 200) return fail(RVE_ENOROOT, "control: bracket search failed");
                lo = hi; flo = fhi; h *= 4.0; hi = lo + h;
                if ((rc = evaluate(hi, fhi))) return rc;
            }
        } else {
            hi = E0; fhi = f0; lo = std::max(0.0, hi - h);
            if ((rc = evaluate(lo, flo))) return rc;
            while (flo >= 0.0) {
                if (lo == 0.0) { E_out = 0.0; return RVE_OK; }
                if (++guard > 200) return fail(RVE_ENOROOT, "control: bracket search (downward) failed");
                hi = lo; fhi = flo; h *= 4.0; lo = std::max(0.0, hi - h);
                if ((rc = evaluate(lo, flo))) return rc;
            }
        }
        return illinois(tau, lo, flo, hi, fhi, evaluate, E_out);
    }
    // Refinement of a bracket f(lo) < 0 < f(hi): a secant step through the two latest evaluations
    // when it falls inside the bracket, else the Illinois step. It also stops when the damage solve
    // at the new E needed no iteration: its warm start (the previous evaluation's phi) already met
    // the solve tolerance, so D cannot be resolved any finer at this tolerance and further steps
    // would only see the same value.
    double root_slope = 0.0;  // dD/dE from the last well-separated pair of evaluations
    int eval_iters = 0;
    template <class Ev>
    int illinois(double tau, double lo, double flo, double hi, double fhi, Ev &evaluate, double &E_out) {
        int side = 0, rc;
        double Ea = lo, fa = flo, Eb = hi, fb = fhi;  // the two latest evaluations
        for (int k = 0; k < cfg.max_root_evals; ++k) {
            double E = (lo * fhi - hi * flo) / (fhi - flo);
            if (fb != fa) {
                const double Es = Eb - fb * (Eb - Ea) / (fb - fa);
                if (Es > lo && Es < hi) E = Es;
            }
            double fE;
            if ((rc = evaluate(E, fE))) return rc;
            Ea = Eb; fa = fb; Eb = E; fb = fE;
            if (std::fabs(fE) <= cfg.tol_root * tau || (hi - lo) <= 1e-15 * hi || eval_iters == 0) {
                E_out = E;
                return RVE_OK;
            }
            if (fE > 0.0) {
                hi = E; fhi = fE;
                if (side == 1) flo *= 0.5;
                side = 1;
            } else {
                lo = E; flo = fE;
                if (side == -1) fhi *= 0.5;
                side = -1;
            }
        }
        return fail(RVE_ENOROOT, "control: no root of D(phi(E)) = tau within the evaluation cap");
    }
    // ---- one increment (a1-a11) ----------------------------------------------------------------
    // One increment with cutback: when the staggered iteration does not converge (snap-back near
    // coalescence), the increment is replaced by two of half the dissipation, recursively up to
    // four levels; each sub-increment is committed as its own point of the load curve.
    bool stag_failed = false, accept_unconverged = false;
    int step(double dtau, rve_step_result *out) override {
        Range nvtx("increment");
        // the Newton scheme needs E > 0 (psi_o is quadratic in E, so at E = 0 the Jacobian has no
        // coupling from E to the damage): the first increment is taken by the staggered solver
        if (cfg.solver == RVE_SOLVER_NEWTON && S.E > 0.0) return step_newton(dtau, out);
        return step_cut(dtau, out, 0);
    }

    // ---- monolithic Newton-Raphson increment (Sec. 4.1) ------------------------------------------
    // Newton on (e, phi, E) with BiCGSTAB for J dq = -R (Eqs. (schemeSys), (aniSystem_CrackLength),
    // (aniCrackLength_linearization)), right-preconditioned on the damage block by the FFT
    // Helmholtz inverse; the shadow residual is a fixed hash vector (with the right-hand side as
    // shadow, the first step divides by ~0: J has no E-E entry). Relaxation of Eq. (relax),
    // stopping test of Eq. (errors_crack) as in the staggered solver. The BiCGSTAB scalars live
    // on the host (one read per reduction); the E components of the vectors too.
    T *nrbuf = nullptr;
    template <class F> void pointwise_n(const F &f, Scal *s, long long n) {
        k_pointwise<F><<<(int)pw_blocks<F>(n), 256, 0, st>>>(n, f, partials, s);
        CK(cudaGetLastError());
        ++launches;
    }
    template <int NSx> NRPoint<T, NSx> nr_point(const T *e, const T *ph, double E) const {
        NRPoint<T, NSx> q{Cm, gid, e, ph, E, {}, cfg.k_res, N};
        for (int a = 0; a < NSx; ++a) q.f[a] = fM[a];
        return q;
    }
    // v -> J v (vectors [e | phi] plus the E component); returns J3 (the E component of J v)
    template <int NSx, int Dx> double nr_apply(const NRPoint<T, NSx> &q, const T *vin, double vE, T *vout) {
        init_sc(sc2, 0.0, 0);
        x_fwd<NSx>(ProNRMech<T, NSx>{false, q, vin, vin + (size_t)NSx * N, vE}, sc2);
        spectral<NSx, NSx>(OpProj<C, NSx>{false, xitab()}, sc2);
        x_inv<NSx>(EpiNRStore<T, NSx>{false, vout, 1.0, N}, sc2);
        x_fwd<1>(ProField<T>{false, vin + (size_t)NSx * N}, sc2);
        spectral<1, Dx>(OpGrad<C, Dx>{false, xitab()}, sc2);
        x_mid<Dx>(MidFlux<T, Dx>{false, Ktab, gid}, sc2);
        spectral<Dx, 1>(OpDiv<C, Dx>{false, xitab()}, sc2);
        x_inv<1>(EpiNRDmg<T, NSx>{false, q, acoef, psi_ini, H, cfg.history, vin, vin + (size_t)NSx * N, vE,
                                  vout + (size_t)NSx * N},
                 sc2);
        read_sc(sc2);
        return h_sc->red[0];
    }
    // b = -R at q; returns -R3 and the norms of R1, R2 and their scales, D and sum H
    struct NRRes { double mR3, nR1, nR2, s1, s2, D, Hsum; };
    template <int NSx, int Dx> NRRes nr_residual(const NRPoint<T, NSx> &q, double tau, T *b) {
        init_sc(sc2, 0.0, 0);
        x_fwd<NSx>(ProNRMech<T, NSx>{false, q, nullptr, nullptr, 0.0}, sc2);
        spectral<NSx, NSx>(OpProj<C, NSx>{false, xitab()}, sc2);
        x_inv<NSx>(EpiNRStore<T, NSx>{false, b, -1.0, N}, sc2);
        x_fwd<1>(ProField<T>{false, q.phi}, sc2);
        spectral<1, Dx>(OpGrad<C, Dx>{false, xitab()}, sc2);
        x_mid<Dx>(MidFlux<T, Dx>{false, Ktab, gid}, sc2);
        spectral<Dx, 1>(OpDiv<C, Dx>{false, xitab()}, sc2);
        x_inv<1>(EpiNRDmg<T, NSx>{false, q, acoef, psi_ini, H, cfg.history, nullptr, nullptr, 0.0,
                                  b + (size_t)NSx * N},
                 sc2);
        read_sc(sc2);
        NRRes r;
        r.nR1 = std::sqrt(h_sc->rr);
        r.s1 = std::sqrt(h_sc->scale2);
        r.nR2 = std::sqrt(h_sc->red[0]);
        r.s2 = std::sqrt(h_sc->red[1]);
        r.D = h_sc->red[2];
        r.Hsum = h_sc->red[3];
        r.mR3 = -(r.D - tau);
        return r;
    }
    // right preconditioner: identity on e and E, (abar + bbar |xi~|^2)^-1 on phi (abar, bbar in sc3)
    void nr_precond(const T *in, T *out) {
        CK(cudaMemcpyAsync(out, in, sizeof(T) * NS * N, cudaMemcpyDeviceToDevice, st));
        x_fwd<1>(ProField<T>{false, in + (size_t)NS * N}, sc3);
        spectral<1, 1>(OpPrec<C>{false, sc3, xitab()}, sc3);
        x_inv<1>(EpiStore<T>{false, out + (size_t)NS * N}, sc3);
    }
    double nr_dot(const T *a, const T *b, long long n) {
        init_sc(sc2, 0.0, 0);
        pointwise_n(PwVDot<T>{false, a, b, nullptr, nullptr}, sc2, n);
        read_sc(sc2);
        return h_sc->red[0];
    }
    void nr_dot2(const T *a, const T *b, const T *c, const T *d, long long n, double &ab, double &cd) {
        init_sc(sc2, 0.0, 0);
        pointwise_n(PwVDot<T>{false, a, b, c, d}, sc2, n);
        read_sc(sc2);
        ab = h_sc->red[0];
        cd = h_sc->red[1];
    }
    void nr_comb(T *out, const T *a, double ca, const T *b, double cb, const T *c, double cc, long long n) {
        pointwise_n(PwVComb<T>{false, out, a, b, c, ca, cb, cc}, sc2, n);
    }
    template <int NSx, int Dx>
    int nr_bicgstab(const NRPoint<T, NSx> &q, const T *b, double bE, double tol, int maxit, T *x, double &xE,
                    int &its) {
        // work vectors: slots 3..10 of nrbuf (0: iterate, 1: right-hand side, 2: solution)
        const long long n = (long long)(NSx + 1) * N;
        T *r = nrbuf + 3 * n, *rh = nrbuf + 4 * n, *p = nrbuf + 5 * n, *v = nrbuf + 6 * n, *s = nrbuf + 7 * n,
          *t = nrbuf + 8 * n, *ph = nrbuf + 9 * n, *sh = nrbuf + 10 * n;
        CK(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
        CK(cudaMemcpyAsync(r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(p, 0, sizeof(T) * n, st));
        CK(cudaMemsetAsync(v, 0, sizeof(T) * n, st));
        pointwise_n(PwVHash<T>{false, rh}, sc2, n);
        double rE = bE, rhE = 1.0, pE = 0.0, vE = 0.0;
        xE = 0.0;
        const double nb = std::sqrt(nr_dot(b, b, n) + bE * bE);
        its = 0;
        if (!(nb > 0.0)) return RVE_OK;
        double rho = 1.0, alpha = 1.0, omega = 1.0, nr_last = nb;
        // a breakdown (rho or omega vanishing) with the residual already small keeps x: in FP32 the
        // recurrences reach the rounding floor of the vectors before a strict tolerance
        auto breakdown = [&]() { return nr_last <= 1e-3 * nb ? RVE_OK : fail(RVE_EBREAKDOWN, "Newton: BiCGSTAB breakdown"); };
        for (int it = 1; it <= maxit; ++it) {
            its = it;
            const double rho_new = nr_dot(rh, r, n) + rhE * rE;
            if (rho_new == 0.0 || !std::isfinite(rho_new)) return breakdown();
            const double beta = (rho_new / rho) * (alpha / omega);
            nr_comb(p, r, 1.0, p, beta, v, -beta * omega, n);  // p = r + beta (p - omega v)
            pE = rE + beta * (pE - omega * vE);
            nr_precond(p, ph);
            const double phE = pE;
            vE = nr_apply<NSx, Dx>(q, ph, phE, v);
            alpha = rho_new / (nr_dot(rh, v, n) + rhE * vE);
            nr_comb(s, r, 1.0, v, -alpha, nullptr, 0.0, n);
            const double sE = rE - alpha * vE;
            const double ns = std::sqrt(nr_dot(s, s, n) + sE * sE);
            if (ns <= tol * nb) {
                nr_comb(x, x, 1.0, ph, alpha, nullptr, 0.0, n);
                xE += alpha * phE;
                return RVE_OK;
            }
            nr_precond(s, sh);
            const double shE = sE;
            const double tE = nr_apply<NSx, Dx>(q, sh, shE, t);
            double ts, tt;
            nr_dot2(t, s, t, t, n, ts, tt);
            ts += tE * sE;
            tt += tE * tE;
            omega = ts / tt;
            if (!std::isfinite(omega) || omega == 0.0) {
                if (ns <= 1e-3 * nb) {
                    nr_comb(x, x, 1.0, ph, alpha, nullptr, 0.0, n);
                    xE += alpha * phE;
                    return RVE_OK;
                }
                return breakdown();
            }
            nr_comb(x, x, 1.0, ph, alpha, sh, omega, n);
            xE += alpha * phE + omega * shE;
            nr_comb(r, s, 1.0, t, -omega, nullptr, 0.0, n);
            rE = sE - omega * tE;
            const double nr = std::sqrt(nr_dot(r, r, n) + rE * rE);
            if (!std::isfinite(nr)) return fail(RVE_EBREAKDOWN, "Newton: BiCGSTAB non-finite residual");
            nr_last = nr;
            if (nr <= tol * nb) return RVE_OK;
            rho = rho_new;
        }
        return fail(RVE_ENOCONV, "Newton: BiCGSTAB iteration cap");
    }
    int step_newton(double dtau, rve_step_result *out) {
        Range nvtx("newton increment");
        if (!micro_set) return RVE_ESTATE;
        if (!(dtau > 0.0)) return RVE_EINVAL;
        return NS == 3 ? (D == 2 ? step_newton_t<3, 2>(dtau, out) : step_newton_t<3, 3>(dtau, out))
                       : step_newton_t<6, 3>(dtau, out);
    }
    template <int NSx, int Dx> int step_newton_t(double dtau, rve_step_result *out) {
        const long long n = (long long)(NSx + 1) * N;
        if (!nrbuf) nrbuf = alloc<T>((size_t)11 * n);
        if (!sc3) sc3 = alloc<Scal>(1);
        T *qv = nrbuf, *b = nrbuf + n, *dq = nrbuf + 2 * n;  // iterate [e | phi], -R, Newton step
        rve_step_result r{};
        const double tau = S.tau + dtau;
        double E = S.E;
        // q_0 = q^n: e = E x (x the committed unit-load fluctuation), phi^n
        nr_comb(qv, mx, E, nullptr, 0.0, nullptr, 0.0, (long long)NSx * N);
        CK(cudaMemcpyAsync(qv + (size_t)NSx * N, phi, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        const double alpha = S.Sigma_max > 0.0 ? std::max(0.3, S.Sigma / S.Sigma_max) : 1.0;
        const double tol_floor = 1e-14;
        double err = 1e300, Dv = 0.0;
        int newton = 0, lin = 0;
        bool converged = false;
        for (int k = 0; k < cfg.max_stag_iters && k < 50; ++k) {
            const NRPoint<T, NSx> q = nr_point<NSx>(qv, qv + (size_t)NSx * N, E);
            const NRRes R = nr_residual<NSx, Dx>(q, tau, b);
            if (!std::isfinite(R.nR1) || !std::isfinite(R.nR2) || !std::isfinite(R.D))
                return fail(RVE_EBREAKDOWN, "Newton: non-finite residual");
            init_sc(sc3, 0.0, 0, si.amean + 2.0 * R.Hsum / (double)N, si.bbar);
            const double tol_lin = std::max(tol_floor, std::min(1e-4, 0.01 * err));
            int its = 0;
            double dE = 0.0;
            int rc = nr_bicgstab<NSx, Dx>(q, b, R.mR3, tol_lin, 4000, dq, dE, its);
            if (rc) return rc;
            lin += its;
            ++newton;
            nr_comb(qv, qv, 1.0, dq, alpha, nullptr, 0.0, n);  // q += alpha dq
            E += alpha * dE;
            // Eq. (errors_crack) at the new point: strain change (degraded energy norm), damage
            // change, control
            const NRPoint<T, NSx> q1 = nr_point<NSx>(qv, qv + (size_t)NSx * N, E);
            nr_comb(dq, dq, alpha, nullptr, 0.0, nullptr, 0.0, n);  // the applied step
            init_sc(sc2, 0.0, 0);
            pointwise(PwNRErr<T, NSx>{false, q1, dq, dq + (size_t)NSx * N, alpha * dE}, sc2);
            read_sc(sc2);
            const double e1 = std::sqrt(std::max(h_sc->red[0], 0.0)) / std::max(std::sqrt(std::max(h_sc->red[1], 0.0)), 1e-300);
            const double e2 = std::sqrt(h_sc->red[2]) / std::max(std::sqrt(h_sc->red[3]), 1e-300);
            double Gm;
            dissipation(qv + (size_t)NSx * N, Dv, Gm);
            err = std::max(std::max(e1, e2), std::fabs(Dv - tau) / tau);
            if (err < cfg.tol_stag) { converged = true; break; }
        }
        r.stag_iters = newton;
        r.mech_iters = lin;  // BiCGSTAB iterations (each applies the coupled Jacobian twice)
        r.stag_err = err;
        if (!converged) {
            char buf[160];
            std::snprintf(buf, sizeof(buf), "Newton-Raphson: %d steps, error %.3e (tol %.1e) at increment %d", newton,
                          err, cfg.tol_stag, S.n + 1);
            g_last_error = buf;
            if (out) *out = r;
            return RVE_ENOCONV;
        }
        // commit: phi, strain, unit-load fluctuation, history, Sigma, E_mec, T
        const NRPoint<T, NSx> q = nr_point<NSx>(qv, qv + (size_t)NSx * N, E);
        CK(cudaMemcpyAsync(phi, qv + (size_t)NSx * N, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(phi_trial, phi, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        pointwise(PwNRHistory<T, NSx>{false, q, psi_ini, H, cfg.history, Hcur}, sc2);
        CK(cudaMemcpyAsync(H, Hcur, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        nr_comb(mx, qv, 1.0 / E, nullptr, 0.0, nullptr, 0.0, (long long)NSx * N);
        F6 f6{};
        for (int a = 0; a < NSx; ++a) f6.f[a] = fM[a];
        k_nr_total_strain<T><<<(int)((N + 255) / 256), 256, 0, st>>>(N, NSx, qv, E, f6, eps_com);
        CK(cudaGetLastError());
        ++launches;
        PwPsi1<T, NSx> ps{false, Cm, mx, gid, psi1, {}, N};
        for (int a = 0; a < NSx; ++a) ps.f[a] = (T)fM[a];
        pointwise(ps, sc2);
        init_sc(sc2, 0, 0);
        PwCommit<T, NSx> pc{false, Cm, mx, phi, psi1, gid, {}, E, cfg.k_res, N};
        for (int a = 0; a < NSx; ++a) pc.f[a] = fM[a];
        pointwise(pc, sc2);
        read_sc(sc2);
        const double Sigma = h_sc->red[4] / (double)N;
        const double Emec = h_sc->red[5];
        double Dc, Gc_;
        dissipation(phi, Dc, Gc_);
        const double dT = 0.5 * (Sigma + S.Sigma) * (E - S.E), dG = Gc_ - S.Gamma;
        r.G_inst = dG != 0.0 ? (double)N * dT / dG : NAN;
        S.T += dT;
        S.D = Dc;
        S.Gamma = Gc_;
        S.Sigma = Sigma;
        S.Sigma_max = std::max(S.Sigma_max, Sigma);
        S.E = E;
        S.tau = tau;
        S.n += 1;
        S.fractured = (S.Sigma_max > 0.0 && Sigma <= cfg.fracture_ratio * S.Sigma_max) ? 1 : 0;
        r.n = S.n; r.E = E; r.Sigma = Sigma; r.D = Dc; r.Emec = Emec; r.T = S.T; r.Gamma = Gc_; r.tau = tau;
        r.fractured = S.fractured;
        curve.push_back(r);
        if (out) *out = r;
        return RVE_OK;
    }
    int step_cut(double dtau, rve_step_result *out, int depth) {
        rve_step_result a{};
        accept_unconverged = false;
        int rc = step_once(dtau, &a);
        if (rc == RVE_ENOCONV && stag_failed && depth >= 4) {
            // deepest level: keep the last staggered iterate, flagged
            accept_unconverged = true;
            rc = step_once(dtau, &a);
            accept_unconverged = false;
        } else if (rc == RVE_ENOCONV && stag_failed) {
            rve_step_result b{}, c{};
            rc = step_cut(0.5 * dtau, &b, depth + 1);
            if (rc) return rc;
            if (!b.fractured) {
                rc = step_cut(0.5 * dtau, &c, depth + 1);
                if (rc) return rc;
            } else {
                c = b;
                std::memset(&b, 0, sizeof(b));
            }
            c.mech_iters += b.mech_iters + a.mech_iters;
            c.dmg_iters += b.dmg_iters + a.dmg_iters;
            c.root_evals += b.root_evals + a.root_evals;
            c.stag_iters += b.stag_iters + a.stag_iters;
            c.flags |= b.flags | RVE_STEP_CUTBACK;
            if (out) *out = c;
            return RVE_OK;
        }
        if (out) *out = a;
        return rc;
    }
    int step_once(double dtau, rve_step_result *out) {
        stag_failed = false;
        if (!micro_set) return RVE_ESTATE;
        rve_step_result r{};
        const double tau = S.tau + dtau;
        if (!(dtau > 0.0)) return RVE_EINVAL;
        CK(cudaMemcpyAsync(phi_cur, phi, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(eps_it, eps_com, sizeof(double) * NS * N, cudaMemcpyDeviceToDevice, st));
        double E = S.E, Dv = 0.0, err = 0.0;
        const int m = std::max(0, std::min(5, cfg.anderson_m));
        std::deque<int> hist;  // slots of (X, G) in chronological order
        int next_slot = 0;
        bool converged = false;
        double best = 1e300;
        int k_best = 0;
        for (int k = 0; k < cfg.max_stag_iters; ++k) {
            int it = 0;
            int rc = mech_solve(phi_cur, it);
            r.mech_iters += it;
            if (rc) return rc;
            CK(cudaMemcpyAsync(phi_trial, phi_cur, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
            rc = arc_length(tau, E, E, Dv, r);
            if (rc) return rc;
            // staggered error, Eq. (errors_crack)
            init_sc(sc2, 0, 0);
            if (NS == 3) {
                PwStagEps<T, 3> pe{false, mx, Cm, phi_cur, gid, eps_it, {}, E, cfg.k_res, N};
                for (int a = 0; a < 3; ++a) pe.f[a] = fM[a];
                pointwise(pe, sc2);
            } else {
                PwStagEps<T, 6> pe{false, mx, Cm, phi_cur, gid, eps_it, {}, E, cfg.k_res, N};
                for (int a = 0; a < 6; ++a) pe.f[a] = fM[a];
                pointwise(pe, sc2);
            }
            pointwise(PwStagPhi<T>{false, phi_trial, phi_cur}, sc2);
            read_sc(sc2);
            const double e1 = std::sqrt(std::max(h_sc->red[0], 0.0)) / std::max(std::sqrt(std::max(h_sc->red[1], 0.0)), 1e-300);
            const double e2 = std::sqrt(h_sc->red[2]) / std::max(std::sqrt(h_sc->red[3]), 1e-300);
            err = std::max(std::max(e1, e2), std::fabs(Dv - tau) / tau);
            r.stag_iters = k + 1;
            if (err < cfg.tol_stag) { converged = true; break; }
            // noise floor: the error has not improved for 20 iterations and is within 1000 x tol
            if (err < best) { best = err; k_best = k; }
            if (k - k_best >= 20 && err <= 1000.0 * cfg.tol_stag) {
                converged = true;
                r.flags |= RVE_STEP_STAGNATED;
                break;
            }
            if (m > 0) {
                // record (X = phi_cur, G = phi_trial), keep the last m + 1
                int slot;
                if ((int)hist.size() < m + 1) slot = next_slot++;
                else { slot = hist.front(); hist.pop_front(); }
                hist.push_back(slot);
                k_copy_cast<T><<<(int)((N + 255) / 256), 256, 0, st>>>(N, phi_cur, xh + (size_t)slot * N);
                k_copy_cast<T><<<(int)((N + 255) / 256), 256, 0, st>>>(N, phi_trial, gh + (size_t)slot * N);
                launches += 2;
                const int K = (int)hist.size() - 1;
                if (K < 1) {
                    CK(cudaMemcpyAsync(phi_cur, phi_trial, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
                } else {
                    AAPtrs hp{};
                    for (int j = 0; j <= K; ++j) {
                        hp.X[j] = xh + (size_t)hist[j] * N;
                        hp.G[j] = gh + (size_t)hist[j] * N;
                    }
                    init_sc(sc2, 0, 0);
                    pointwise(PwAAGram<T>{false, hp, K}, sc2);
                    read_sc(sc2);
                    double M[25], b[5], gam[5];
                    int idx = 0;
                    double full[5][5];
                    for (int a = 0; a < 5; ++a)
                        for (int bb = a; bb < 5; ++bb) { full[a][bb] = full[bb][a] = h_sc->red[idx]; ++idx; }
                    for (int a = 0; a < K; ++a) {
                        for (int bb = 0; bb < K; ++bb) M[a * K + bb] = full[a][bb];
                        b[a] = h_sc->red[15 + a];
                    }
                    pinv_solve(K, M, b, 1e-10, gam);
                    PwAAMix<T> mixf{false, hp, K, {}, phi_cur};
                    for (int a = 0; a < K; ++a) mixf.gam[a] = gam[a];
                    pointwise(mixf, sc2);
                }
            } else {
                CK(cudaMemcpyAsync(phi_cur, phi_trial, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
            }
        }
        if (!converged && accept_unconverged) {
            converged = true;
            r.flags |= RVE_STEP_UNCONVERGED;
        }
        if (!converged) {
            stag_failed = true;
            if (out) *out = r;
            char buf[160];
            std::snprintf(buf, sizeof(buf), "staggered iteration: %d iterations, error %.3e (tol %.1e) at increment %d",
                          cfg.max_stag_iters, err, cfg.tol_stag, S.n + 1);
            g_last_error = buf;
            return RVE_ENOCONV;
        }
        // commit (a8, a11): phi, H, strain, Sigma, E_mec, T
        CK(cudaMemcpyAsync(phi, phi_trial, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(H, Hcur, sizeof(T) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(eps_com, eps_it, sizeof(double) * NS * N, cudaMemcpyDeviceToDevice, st));
        init_sc(sc2, 0, 0);
        if (cfg.split == RVE_SPLIT_SPECTRAL) {
            PwCommitSplit<T> pc{false, mx, phi, lamT, muT, gid, {}, E, cfg.k_res, N};
            for (int a = 0; a < 3; ++a) pc.f[a] = fM[a];
            pointwise(pc, sc2);
        } else if (NS == 3) {
            PwCommit<T, 3> pc{false, Cm, mx, phi, psi1, gid, {}, E, cfg.k_res, N};
            for (int a = 0; a < 3; ++a) pc.f[a] = fM[a];
            pointwise(pc, sc2);
        } else {
            PwCommit<T, 6> pc{false, Cm, mx, phi, psi1, gid, {}, E, cfg.k_res, N};
            for (int a = 0; a < 6; ++a) pc.f[a] = fM[a];
            pointwise(pc, sc2);
        }
        read_sc(sc2);
        const double Sigma = h_sc->red[4] / (double)N;
        const double Emec = h_sc->red[5];
        double Dc, Gc_;
        dissipation(phi, Dc, Gc_);
        const double dT = 0.5 * (Sigma + S.Sigma) * (E - S.E), dG = Gc_ - S.Gamma;
        r.G_inst = dG != 0.0 ? (double)N * dT / dG : NAN;  // Eq. (Gmed)
        S.T += dT;
        S.D = Dc;
        S.Gamma = Gc_;
        S.Sigma = Sigma;
        S.Sigma_max = std::max(S.Sigma_max, Sigma);
        S.E = E;
        S.tau = tau;
        S.n += 1;
        S.fractured = (S.Sigma_max > 0.0 && Sigma <= cfg.fracture_ratio * S.Sigma_max) ? 1 : 0;
        r.n = S.n; r.E = E; r.Sigma = Sigma; r.D = Dc; r.Emec = Emec; r.T = S.T; r.Gamma = Gc_; r.tau = tau;
        r.fractured = S.fractured; r.stag_err = err;
        curve.push_back(r);
        if (out) *out = r;
        return RVE_OK;
    }

    template <typename U> struct PwSum {
        static constexpr int NR = 1;
        static constexpr bool MAXRED = false;
        bool skip_if_done;
        const U *f;
        __device__ void apply(long long v, double *acc) const { acc[0] += (double)f[v]; }
        struct Fin {
            Scal *sc;
            __device__ void operator()(const double *t) const { sc->red[0] = t[0]; }
        };
        __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
    };


    // ---- services of the C ABI ------------------------------------------------------------------
    int mech_solve_committed(int &iters) override {
        int rc = mech_solve(phi, iters);
        CK(cudaStreamSynchronize(st));
        return rc;
    }
    int damage_eval_api(double E, double &Dv, int &iters) override {
        ddiv_ok = false;
        prev_ok = false;
        return damage_eval(E, Dv, iters);
    }
    int dissipation_host(const double *phi_host, double &Dv, double &Gv) override {
        CK(cudaMemcpyAsync(dtmp, phi_host, N * sizeof(double), cudaMemcpyHostToDevice, st));
        k_cast_copy<T><<<(int)((N + 255) / 256), 256, 0, st>>>(N, dtmp, tmpf);
        ++launches;
        dissipation(tmpf, Dv, Gv);
        return RVE_OK;
    }
    // checkpoint payload: phi, H, psi_ini, strain fluctuation (field precision), committed strain
    // (FP64), and the control search's slope memory (so a restored run repeats the same iterates)
    size_t state_bytes() const override {
        return (size_t)N * sizeof(T) * (3 + NS) + (size_t)NS * N * sizeof(double) * (kSingle ? 2 : 1) + sizeof(double);
    }
    void save_state(char *p) override {
        const void *src[5] = {phi, H, psi_ini, mx, eps_com};
        const size_t sz[5] = {N * sizeof(T), N * sizeof(T), N * sizeof(T), NS * N * sizeof(T), NS * N * sizeof(double)};
        for (int i = 0; i < 5; ++i) { CK(cudaMemcpyAsync(p, src[i], sz[i], cudaMemcpyDeviceToHost, st)); p += sz[i]; }
        if (kSingle) {  // the FP64 fluctuation of the refinement, so that a restore continues bit for bit
            ensure_mx64();
            CK(cudaMemcpyAsync(p, mx64, NS * N * sizeof(double), cudaMemcpyDeviceToHost, st));
            p += NS * N * sizeof(double);
        }
        std::memcpy(p, &root_slope, sizeof(double));
        CK(cudaStreamSynchronize(st));
    }
    void load_state(const char *p) override {
        void *dst[5] = {phi, H, psi_ini, mx, eps_com};
        const size_t sz[5] = {N * sizeof(T), N * sizeof(T), N * sizeof(T), NS * N * sizeof(T), NS * N * sizeof(double)};
        for (int i = 0; i < 5; ++i) { CK(cudaMemcpyAsync(dst[i], p, sz[i], cudaMemcpyHostToDevice, st)); p += sz[i]; }
        if (kSingle) {
            if (!mx64) mx64 = alloc<double>((size_t)NS * N);
            CK(cudaMemcpyAsync(mx64, p, NS * N * sizeof(double), cudaMemcpyHostToDevice, st));
            p += NS * N * sizeof(double);
            mx64_ok = true;
        }
        std::memcpy(&root_slope, p, sizeof(double));
        CK(cudaMemcpyAsync(phi_trial, phi, N * sizeof(T), cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    void timing_reset() override { ev_used = 0; }
    void timing_get(int kind, double &ms, long &n, double &bytes, double &flops) override {
        CK(cudaStreamSynchronize(st));
        double tot = 0.0, by = 0.0, fl = 0.0;
        long cnt = 0;
        for (size_t i = 0; i < ev_used; ++i) {
            const EvMeta &m = ev_meta[i];
            const bool take = kind == 0   ? m.sub == 1
                              : kind == 8 ? m.sub == 2
                              : kind == 9 ? m.sub == 3
                              : kind == 6 ? true
                                          : m.kind == kind;  // 7: FP64 residual passes
            if (!take) continue;
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ev_pool[i].first, ev_pool[i].second));
            tot += t;
            by += m.bytes;
            fl += m.flops;
            ++cnt;
        }
        ms = tot;
        n = cnt;
        bytes = cnt ? by / (double)cnt : 0.0;
        flops = cnt ? fl / (double)cnt : 0.0;
    }

    // ---- field access --------------------------------------------------------------------------
    int get_field(int field, double *host, size_t n) override {
        const size_t nsc = (size_t)N, nten = (size_t)NS * N;
        const int blocks = (int)((N + 255) / 256);
        switch (field) {
        case RVE_FIELD_PHI: case RVE_FIELD_H: case RVE_FIELD_PSI_INI: case RVE_FIELD_PSI1: case RVE_FIELD_PHI_TRIAL: {
            if (n != nsc) return RVE_EINVAL;
            const T *src = field == RVE_FIELD_PHI ? phi : field == RVE_FIELD_H ? H : field == RVE_FIELD_PSI_INI ? psi_ini
                         : field == RVE_FIELD_PSI1 ? psi1 : phi_trial;
            k_copy_cast<T><<<blocks, 256, 0, st>>>(N, src, dtmp);
            break;
        }
        case RVE_FIELD_EPS: case RVE_FIELD_SIGMA: case RVE_FIELD_FLUCT1: {
            if (n != nten) return RVE_EINVAL;
            if (field == RVE_FIELD_FLUCT1) {
                k_mandel_to_tensor<T><<<blocks, 256, 0, st>>>(N, D, mx, 1.0, nullptr, dtmp);
            } else if (field == RVE_FIELD_EPS) {
                k_mandel_to_tensor<double><<<blocks, 256, 0, st>>>(N, D, eps_com, 1.0, nullptr, dtmp);
            } else {
                double *sig = alloc_tmp_sig();
                if (cfg.split == RVE_SPLIT_SPECTRAL)
                    k_stress_split<T><<<blocks, 256, 0, st>>>(N, lamT, muT, gid, phi, cfg.k_res, eps_com, sig);
                else
                    k_stress<T><<<blocks, 256, 0, st>>>(N, D, Cm, gid, phi, cfg.k_res, eps_com, sig);
                k_mandel_to_tensor<double><<<blocks, 256, 0, st>>>(N, D, sig, 1.0, nullptr, dtmp);
            }
            break;
        }
        default: return RVE_EINVAL;
        }
        CK(cudaMemcpyAsync(host, dtmp, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return RVE_OK;
    }
    double *sig_tmp = nullptr;
    double *alloc_tmp_sig() {
        if (!sig_tmp) sig_tmp = alloc<double>((size_t)NS * N);
        return sig_tmp;
    }
    int set_field(int field, const double *host, size_t n) override {
        const size_t nsc = (size_t)N, nten = (size_t)NS * N;
        const int blocks = (int)((N + 255) / 256);
        if (field == RVE_FIELD_PHI || field == RVE_FIELD_H || field == RVE_FIELD_PSI_INI) {
            if (n != nsc) return RVE_EINVAL;
            CK(cudaMemcpyAsync(dtmp, host, n * sizeof(double), cudaMemcpyHostToDevice, st));
            T *dst = field == RVE_FIELD_PHI ? phi : field == RVE_FIELD_H ? H : psi_ini;
            k_cast_copy<T><<<blocks, 256, 0, st>>>(N, dtmp, dst);
            if (field == RVE_FIELD_PHI) k_cast_copy<T><<<blocks, 256, 0, st>>>(N, dtmp, phi_trial);
        } else if (field == RVE_FIELD_FLUCT1 || field == RVE_FIELD_EPS) {
            if (n != nten) return RVE_EINVAL;
            CK(cudaMemcpyAsync(dtmp, host, n * sizeof(double), cudaMemcpyHostToDevice, st));
            if (field == RVE_FIELD_FLUCT1) {
                k_tensor_to_mandel<T><<<blocks, 256, 0, st>>>(N, D, dtmp, mx);
                mx64_ok = false;
            }
            else k_tensor_to_mandel<double><<<blocks, 256, 0, st>>>(N, D, dtmp, eps_com);
        } else {
            return RVE_EINVAL;
        }
        CK(cudaStreamSynchronize(st));
        return RVE_OK;
    }
};

// Engine factories, one per field precision, each compiled in a translation unit of its own.
EngineBase *make_engine_f64(const rve_config &c);
EngineBase *make_engine_f32(const rve_config &c);

}  // namespace pffeng
