// Shared device helpers of the FFT phase-field-fracture library (sm_103a).
//
//  * complex arithmetic on double2 / float2,
//  * deterministic block reductions: warp shuffles, then a block tree, then a "last block done"
//    pass that sums the per-block partials in a fixed order (no floating-point atomics), so a
//    reduction gives the same bits for the same launch shape,
//  * an in-place Stockham FFT (radix 4, one radix-2 stage for odd log2 L) over several lines of
//    length L held in shared memory, one register-staged stage per barrier pair.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace pff {

template <typename T> struct cplx_of;
template <> struct cplx_of<double> { typedef double2 type; };
template <> struct cplx_of<float> { typedef float2 type; };
template <typename C> struct real_of;
template <> struct real_of<double2> { typedef double type; };
template <> struct real_of<float2> { typedef float type; };

// Load of a field that no thread of the running kernel writes before reading it (each voxel is
// read, then possibly rewritten, by the one thread that owns it). The read-only path lets the
// compiler issue the loads of several voxels ahead of the stores of earlier ones, instead of
// serialising every voxel behind a possibly aliasing store.
template <typename T> __device__ __forceinline__ T ldro(const T *p) { return __ldg(p); }

template <typename C> __device__ __forceinline__ C cmk(double re, double im) {
    C r; r.x = re; r.y = im; return r;
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }   // i a
__device__ __forceinline__ double2 cmulmi(double2 a) { return make_double2(a.y, -a.x); }  // -i a

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 cmulmi(float2 a) { return make_float2(a.y, -a.x); }

// ---------------------------------------------------------------------------------------------
// Grid geometry and the spectral layout.
//   real fields:     [comp][z][y][x], N = nx ny nz voxels per component
//   half spectrum:   [comp][z][y][kx], kx < Px (Px >= nx/2 + 1, padded to the column tile)
// ---------------------------------------------------------------------------------------------
struct Geom {
    int d, ns;            // spatial dimension, symmetric tensor components (3 or 6)
    int nx, ny, nz;
    int lx, ly, lz;       // log2 of the extents
    int Px;               // spectral pitch (complex elements per row)
    long long N;          // voxels
    long long Nh;         // complex elements per spectral component (Px ny nz)
    double invN;
};

// Device scalars of one iterative solve. All solver control that the GPU needs between kernels
// lives here; the host reads it back once a solve (one graph launch) has finished.
struct Scal {
    double rr, rr0, rz, pq, alpha, beta, scale2;
    double abar, bbar, D, Gamma, red[24];
    int done, iters, flag, first, max_iters, pad_;
    double tol2;
    double eta2;  // inner stop of a refinement pass: <r, r> <= eta2 <r0, r0> (0: none)
    unsigned int counter;
};

enum { FLAG_BREAKDOWN = 1, FLAG_NONFINITE = 2 };

// ---------------------------------------------------------------------------------------------
// Deterministic reductions
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block-reduce NR values (sum), store per-block partials, and let the last block to finish sum
// the partials in block order and call fin(totals) on thread 0. Must be called by all threads.
// partials holds NR * nblocks doubles; sc->counter must be 0 on entry and is reset on exit.
template <int NR, class Fin>
__device__ __forceinline__ void reduce_finalize(double (&v)[NR], double *partials, Scal *sc, Fin fin,
                                                bool use_max = false) {
    __shared__ double sh[NR][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    const unsigned nb = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.x + gridDim.x * blockIdx.y;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        double t = use_max ? warp_max(v[k]) : warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = t;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double t = (lane < nw) ? sh[k][lane] : (use_max ? -1e300 : 0.0);
            t = use_max ? warp_max(t) : warp_sum(t);
            if (lane == 0) partials[(size_t)k * nb + bid] = t;
        }
        if (lane == 0) {
            __threadfence();
            unsigned prev = atomicAdd(&sc->counter, 1u);
            last = (prev == nb - 1);
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // Last block: every thread combines the partials b = tid, tid + blockDim, ... in that order
    // (L2 loads, independent of each other, so they are all in flight at once), then the block
    // combines the threads in a fixed tree. The order is fixed, so the result is deterministic.
    double loc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) loc[k] = use_max ? -1e300 : 0.0;
    for (unsigned b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            const double p = __ldcg(partials + (size_t)k * nb + b);
            loc[k] = use_max ? fmax(loc[k], p) : loc[k] + p;
        }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const double t = use_max ? warp_max(loc[k]) : warp_sum(loc[k]);
        if (lane == 0) sh[k][wid] = t;
    }
    __syncthreads();
    if (wid == 0) {
        double tot[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            double t = (lane < nw) ? sh[k][lane] : (use_max ? -1e300 : 0.0);
            tot[k] = use_max ? warp_max(t) : warp_sum(t);
        }
        if (lane == 0) {
            fin(tot);
            sc->counter = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Shared-memory Stockham FFT.
// Lines of length L = 2^logL (L >= 4) live in shared memory at s + line * L. The CTA has
// TL = L/4 threads per line group; thread tid works on group g = tid / TL and, inside it, on the
// lines  g * grp_stride + i * comp_stride, i < nl (nl <= NL). Every thread of the CTA must call
// this function (it contains barriers). tw[m] = exp(-2 pi i m / L); inv selects exp(+...).
// Stage (radix R, span Ns): butterfly j reads x[j + r L/R], twiddles by w^(r (j mod Ns)) with
// w = exp(-+2 pi i / (Ns R)), applies the R-point DFT and writes y[(j - j mod Ns) R + j mod Ns + q Ns].
// ---------------------------------------------------------------------------------------------
template <typename C, int NL>
__device__ __forceinline__ void fft_lines(C *s, int L, int logL, int nl, int grp_stride, int comp_stride,
                                          const C *__restrict__ tw, bool inv) {
    const int TL = L >> 2;
    const int g = threadIdx.x / TL;
    const int t = threadIdx.x - g * TL;
    int Ns = 1;
    if (logL & 1) {
        C v[NL][2][2];
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            if (i < nl) {
                C *base = s + (size_t)(g * grp_stride + i * comp_stride) * L;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    int j = t + b * TL;
                    v[i][b][0] = base[j];
                    v[i][b][1] = base[j + (L >> 1)];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            if (i < nl) {
                C *base = s + (size_t)(g * grp_stride + i * comp_stride) * L;
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    int j = t + b * TL;
                    base[2 * j] = cadd(v[i][b][0], v[i][b][1]);
                    base[2 * j + 1] = csub(v[i][b][0], v[i][b][1]);
                }
            }
        }
        __syncthreads();
        Ns = 2;
    }
    while (Ns < L) {
        const int k = t & (Ns - 1);
        const int tstride = L / (Ns * 4);
        const int tw1 = k * tstride;
        C w1 = tw[tw1], w2 = tw[2 * tw1], w3 = tw[3 * tw1];
        if (inv) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; }
        C v[NL][4];
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            if (i < nl) {
                C *base = s + (size_t)(g * grp_stride + i * comp_stride) * L;
                v[i][0] = base[t];
                v[i][1] = base[t + TL];
                v[i][2] = base[t + 2 * TL];
                v[i][3] = base[t + 3 * TL];
            }
        }
        __syncthreads();
        const int ob = ((t - k) << 2) + k;
#pragma unroll
        for (int i = 0; i < NL; ++i) {
            if (i < nl) {
                C a0 = v[i][0], a1 = cmul(v[i][1], w1), a2 = cmul(v[i][2], w2), a3 = cmul(v[i][3], w3);
                C p = cadd(a0, a2), m = csub(a0, a2), q = cadd(a1, a3), r = csub(a1, a3);
                C *base = s + (size_t)(g * grp_stride + i * comp_stride) * L;
                base[ob] = cadd(p, q);
                base[ob + 2 * Ns] = csub(p, q);
                if (!inv) {
                    base[ob + Ns] = cadd(m, cmulmi(r));
                    base[ob + 3 * Ns] = cadd(m, cmuli(r));
                } else {
                    base[ob + Ns] = cadd(m, cmuli(r));
                    base[ob + 3 * Ns] = cadd(m, cmulmi(r));
                }
            }
        }
        __syncthreads();
        Ns <<= 2;
    }
}

// Frequency of index k on an axis of n points (FFT order), Nyquist set to zero.
__device__ __forceinline__ double xi_of(int k, int n) {
    int kk = (k <= (n >> 1)) ? k : k - n;
    if (2 * k == n) return 0.0;
    return 6.283185307179586476925286766559 * (double)kk / (double)n;
}

}  // namespace pff
