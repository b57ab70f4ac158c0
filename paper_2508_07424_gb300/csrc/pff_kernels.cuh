// Fused spectral passes of the FFT phase-field-fracture solver (sm_103a).
//
// A spectral operator  v -> F^-1[ Op(xi) F[ pro(v) ] ]  is applied as
//   k_x_fwd   : per pair of x-rows, evaluate the prologue (e.g. the stress C_phi : p of a CG
//               direction) for NC components, pack the two real rows as one complex line, FFT
//               along x in shared memory, split into the two half spectra, store [c][z][y][kx];
//   k_axis    : per tile of CW adjacent kx columns, FFT along y (2D) or y then z (3D), one warp
//               per line in registers, apply the per-frequency operator (projection, gradient,
//               divergence, preconditioner), inverse FFT, store;
//   k_x_inv   : rebuild the packed line from two half spectra, inverse FFT along x, evaluate the
//               epilogue (CG vector update, residual, dot products) with a deterministic
//               reduction finalised by the last CTA.
//   k_x_mid   : inverse x pass, a pointwise map (damage flux Gc l A grad phi), forward x pass.
// All kernels of one solve read their scalars (alpha, beta, done flag) from a device Scal block,
// so a whole CG iteration is launched without host synchronisation.
#pragma once

#include <type_traits>

#include "pff_common.cuh"

namespace pff {

enum { AX_FWD = 0, AX_INV = 1, AX_FWD_OP_INV = 2 };

// Epilogues that define FACC = true also provide apply_f(v, val, float *acc), used on the FP32
// path to accumulate a thread's partial sums in FP32.
template <class E, class = void> struct facc_of : std::false_type {};
template <class E> struct facc_of<E, std::void_t<decltype(E::FACC)>> : std::integral_constant<bool, E::FACC> {};

// Launch bounds of the forward x pass: at most 256 threads (max(128, nx / 4)); on the FP32 path
// at least 3 such CTAs per SM (<= 85 registers), so that more warps cover the latency of the
// fused prologue's loads, which bound it on large grids (128^3: 174 -> 150 us per CG launch;
// the inverse and middle x passes measured 5-10 % slower with the same bound and keep theirs).
template <typename T> __host__ __device__ constexpr int x_max_threads() { return sizeof(T) == 4 ? 256 : 512; }
template <typename T> __host__ __device__ constexpr int x_min_blocks() { return sizeof(T) == 4 ? 3 : 1; }

// ---- x-axis forward (r2c) pass ------------------------------------------------------------------
template <typename T, int NC, class Pro>
__device__ __forceinline__ void x_fwd_body(const Geom &g, const Pro &pro, typename cplx_of<T>::type *__restrict__ spec,
                                           const typename cplx_of<T>::type *__restrict__ tw, double *partials,
                                           Scal *sc) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    if (pro.skip_if_done && sc->done) return;
    const int nx = g.nx, TL = nx >> 2;
    const int rp = threadIdx.x / TL, t = threadIdx.x - rp * TL;
    const int RP = blockDim.x / TL;
    const long long pair = (long long)blockIdx.x * RP + rp;
    const int ppp = g.ny >> 1;
    const int z = (int)(pair / ppp), y0 = 2 * (int)(pair % ppp);
    const long long row0 = ((long long)z * g.ny + y0) * nx;
    double acc[Pro::NR > 0 ? Pro::NR : 1];
#pragma unroll
    for (int k = 0; k < (Pro::NR > 0 ? Pro::NR : 1); ++k) acc[k] = 0.0;
    C *line = s + (size_t)rp * NC * nx;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = t + q * TL;
        T va[NC], vb[NC];
        pro.eval(row0 + x, va, acc);
        pro.eval(row0 + nx + x, vb, acc);
#pragma unroll
        for (int c = 0; c < NC; ++c) line[c * nx + x] = cmk<C>(va[c], vb[c]);
    }
    __syncthreads();
    fft_lines<C, NC>(s, nx, g.lx, NC, NC, 1, tw, false);
    const int nh = (nx >> 1) + 1;
    for (int k = t; k < nh; k += TL) {
        const int km = (nx - k) & (nx - 1);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const C Z = line[c * nx + k], Zm = line[c * nx + km];
            C Xa, Xb;
            Xa.x = (T)0.5 * (Z.x + Zm.x);
            Xa.y = (T)0.5 * (Z.y - Zm.y);
            Xb.x = (T)0.5 * (Z.y + Zm.y);
            Xb.y = (T)-0.5 * (Z.x - Zm.x);
            C *dst = spec + (size_t)c * g.Nh + ((long long)z * g.ny + y0) * g.Px + k;
            dst[0] = Xa;
            dst[g.Px] = Xb;
        }
    }
    if constexpr (Pro::NR > 0) reduce_finalize<Pro::NR>(acc, partials, sc, pro.fin(sc));
}

template <typename T, int NC, class Pro>
__global__ void __launch_bounds__(x_max_threads<T>(), x_min_blocks<T>()) k_x_fwd(Geom g, Pro pro, typename cplx_of<T>::type *__restrict__ spec,
                                               const typename cplx_of<T>::type *__restrict__ tw, double *partials,
                                               Scal *sc) {
    x_fwd_body<T, NC>(g, pro, spec, tw, partials, sc);
}

// ---- batched launches: several RVEs of one grid in one launch -----------------------------------
// blockIdx.z selects the RVE; each carries its own functor, spectral buffer, reduction partials
// and scalar block (the per-RVE reductions see gridDim.x * gridDim.y blocks, as unbatched).
constexpr int kMaxBatch = 16;
template <class F> struct SlotArg {
    F f;
    void *spec;
    double *partials;
    Scal *sc;
};
template <class F> struct SlotArgs {
    SlotArg<F> a[kMaxBatch];
};

template <typename T, int NC, class Pro>
__global__ void __launch_bounds__(x_max_threads<T>(), x_min_blocks<T>()) k_x_fwd_b(Geom g, SlotArgs<Pro> args,
                                                 const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    const SlotArg<Pro> &a = args.a[blockIdx.z];
    x_fwd_body<T, NC>(g, a.f, (C *)a.spec, tw, a.partials, a.sc);
}

// Load the packed complex line Z = Xa + i Xb of rows (y0, y0+1) from the half spectra.
template <typename T, typename C>
__device__ __forceinline__ void load_packed(const Geom &g, const C *__restrict__ spec, int c, int z, int y0,
                                            C *line, int t, int TL) {
    const int nx = g.nx, nh2 = nx >> 1;
    const C *src = spec + (size_t)c * g.Nh + ((long long)z * g.ny + y0) * g.Px;
    // TL = nx / 4, so k = t, t + TL and (for t = 0 only) t + 2 TL = nx / 2; a fixed trip count
    // lets the loads of all three be issued together
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int k = t + q * TL;
        if (k > nh2) break;
        C Xa = src[k], Xb = src[g.Px + k];
        if (k == 0 || k == nh2) { Xa.y = 0; Xb.y = 0; }
        C Z;
        Z.x = Xa.x - Xb.y;
        Z.y = Xa.y + Xb.x;
        line[k] = Z;
        if (k > 0 && k < nh2) {
            C Zc;
            Zc.x = Xa.x + Xb.y;
            Zc.y = -Xa.y + Xb.x;
            line[nx - k] = Zc;
        }
    }
}

// ---- x-axis inverse (c2r) pass with a fused epilogue --------------------------------------------
template <typename T, int NC, class Epi>
__device__ __forceinline__ void x_inv_body(const Geom &g, const typename cplx_of<T>::type *__restrict__ spec,
                                           const Epi &epi, const typename cplx_of<T>::type *__restrict__ tw,
                                           double *partials, Scal *sc) {
    typedef typename cplx_of<T>::type C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    if (epi.skip_if_done && sc->done) return;
    const int nx = g.nx, TL = nx >> 2;
    const int rp = threadIdx.x / TL, t = threadIdx.x - rp * TL;
    const int RP = blockDim.x / TL;
    const long long pair = (long long)blockIdx.x * RP + rp;
    const int ppp = g.ny >> 1;
    const int z = (int)(pair / ppp), y0 = 2 * (int)(pair % ppp);
    const long long row0 = ((long long)z * g.ny + y0) * nx;
    C *line = s + (size_t)rp * NC * nx;
#pragma unroll
    for (int c = 0; c < NC; ++c) load_packed<T, C>(g, spec, c, z, y0, line + c * nx, t, TL);
    __syncthreads();
    fft_lines<C, NC>(s, nx, g.lx, NC, NC, 1, tw, true);
    constexpr int NR1 = Epi::NR > 0 ? Epi::NR : 1;
    double acc[NR1];
#pragma unroll
    for (int k = 0; k < NR1; ++k) acc[k] = 0.0;
    const T sN = (T)g.invN;
    // FP32 path with an epilogue that supports it: the thread's 8 voxels are summed in FP32 and
    // converted once (FP64 issues at 1/64 of the FP32 rate on this part); the reduction across
    // threads and CTAs stays FP64
    constexpr bool F32ACC = sizeof(T) == 4 && facc_of<Epi>::value;
    float accf[NR1];
#pragma unroll
    for (int k = 0; k < NR1; ++k) accf[k] = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = t + q * TL;
        T va[NC], vb[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const C v = line[c * nx + x];
            va[c] = v.x * sN;
            vb[c] = v.y * sN;
        }
        if constexpr (F32ACC) {
            epi.apply_f(row0 + x, va, accf);
            epi.apply_f(row0 + nx + x, vb, accf);
        } else {
            epi.apply(row0 + x, va, acc);
            epi.apply(row0 + nx + x, vb, acc);
        }
    }
    if constexpr (F32ACC) {
#pragma unroll
        for (int k = 0; k < NR1; ++k) acc[k] = (double)accf[k];
    }
    if constexpr (Epi::NR > 0) reduce_finalize<Epi::NR>(acc, partials, sc, epi.fin(sc));
}

template <typename T, int NC, class Epi>
__global__ void __launch_bounds__(512) k_x_inv(Geom g, const typename cplx_of<T>::type *__restrict__ spec, Epi epi,
                                               const typename cplx_of<T>::type *__restrict__ tw, double *partials,
                                               Scal *sc) {
    x_inv_body<T, NC>(g, spec, epi, tw, partials, sc);
}

template <typename T, int NC, class Epi>
__global__ void __launch_bounds__(512) k_x_inv_b(Geom g, SlotArgs<Epi> args,
                                                 const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    const SlotArg<Epi> &a = args.a[blockIdx.z];
    x_inv_body<T, NC>(g, (const C *)a.spec, a.f, tw, a.partials, a.sc);
}

// ---- x-axis inverse, pointwise map, x-axis forward ----------------------------------------------
// Inverse x pass of NCI components, mid.apply(v, in[NCI], out[NCO]) per voxel (NCO <= NCI), forward
// x pass of the NCO outputs.
template <typename T, int NCI, int NCO, class Mid>
__device__ __forceinline__ void x_mid_body(const Geom &g, typename cplx_of<T>::type *__restrict__ spec, const Mid &mid,
                                           const typename cplx_of<T>::type *__restrict__ tw, Scal *sc) {
    typedef typename cplx_of<T>::type C;
    static_assert(NCO <= NCI, "k_x_mid maps NCI components to at most NCI");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    if (mid.skip_if_done && sc->done) return;
    const int nx = g.nx, TL = nx >> 2;
    const int rp = threadIdx.x / TL, t = threadIdx.x - rp * TL;
    const int RP = blockDim.x / TL;
    const long long pair = (long long)blockIdx.x * RP + rp;
    const int ppp = g.ny >> 1;
    const int z = (int)(pair / ppp), y0 = 2 * (int)(pair % ppp);
    const long long row0 = ((long long)z * g.ny + y0) * nx;
    C *line = s + (size_t)rp * NCI * nx;
#pragma unroll
    for (int c = 0; c < NCI; ++c) load_packed<T, C>(g, spec, c, z, y0, line + c * nx, t, TL);
    __syncthreads();
    fft_lines<C, NCI>(s, nx, g.lx, NCI, NCI, 1, tw, true);
    const T sN = (T)g.invN;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = t + q * TL;
        T va[NCI], vb[NCI], oa[NCO], ob[NCO];
#pragma unroll
        for (int c = 0; c < NCI; ++c) {
            const C v = line[c * nx + x];
            va[c] = v.x * sN;
            vb[c] = v.y * sN;
        }
        mid.apply(row0 + x, va, oa);
        mid.apply(row0 + nx + x, vb, ob);
#pragma unroll
        for (int c = 0; c < NCO; ++c) line[c * nx + x] = cmk<C>(oa[c], ob[c]);
    }
    __syncthreads();
    fft_lines<C, NCI>(s, nx, g.lx, NCO, NCI, 1, tw, false);
    const int nh = (nx >> 1) + 1;
    for (int k = t; k < nh; k += TL) {
        const int km = (nx - k) & (nx - 1);
#pragma unroll
        for (int c = 0; c < NCO; ++c) {
            const C Z = line[c * nx + k], Zm = line[c * nx + km];
            C Xa, Xb;
            Xa.x = (T)0.5 * (Z.x + Zm.x);
            Xa.y = (T)0.5 * (Z.y - Zm.y);
            Xb.x = (T)0.5 * (Z.y + Zm.y);
            Xb.y = (T)-0.5 * (Z.x - Zm.x);
            C *dst = spec + (size_t)c * g.Nh + ((long long)z * g.ny + y0) * g.Px + k;
            dst[0] = Xa;
            dst[g.Px] = Xb;
        }
    }
}

template <typename T, int NCI, int NCO, class Mid>
__global__ void __launch_bounds__(512) k_x_mid(Geom g, typename cplx_of<T>::type *__restrict__ spec, Mid mid,
                                               const typename cplx_of<T>::type *__restrict__ tw, Scal *sc) {
    x_mid_body<T, NCI, NCO>(g, spec, mid, tw, sc);
}

template <typename T, int NCI, int NCO, class Mid>
__global__ void __launch_bounds__(512) k_x_mid_b(Geom g, SlotArgs<Mid> args,
                                                 const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    const SlotArg<Mid> &a = args.a[blockIdx.z];
    x_mid_body<T, NCI, NCO>(g, (C *)a.spec, a.f, tw, a.sc);
}


// ---- y / z axis pass ----------------------------------------------------------------------------
// axis = 1 (y) or 2 (z). A CTA owns CW adjacent kx columns of one plane (z for axis y, y for
// axis z) and all L points along the axis, for every component. MODE: AX_FWD, AX_INV or
// AX_FWD_OP_INV (forward, the per-frequency operator mapping NCI -> NCO components, inverse).
//
//  1. The tile is read from global memory with consecutive threads on consecutive kx (coalesced
//     runs of CW complex values per row) into shared memory, one line of L points per
//     (component, column). Lines are padded so that the transposing writes hit distinct banks.
//  2. Each line is transformed by one warp (or a lane group of S = L / R lanes when L < 128) in
//     registers: lane l holds the R points l + S m (m < R); an R-point decimation-in-frequency
//     FFT over m, a twiddle by w_L^(l k1), then an S-point DIF across the lanes with shuffles
//     (see wfft_fwd). No CTA barrier is taken inside a transform. The spectrum is left in the
//     scrambled storage order of the network: position p = l + S m holds the frequency
//     axis_freq(p) = brev_R(m) + R brev_S(l); the operator is evaluated there, and the inverse
//     network (wfft_inv) takes that order back to natural order. In 3D the y pass stores its
//     spectrum in storage order between the forward and the inverse y passes, so the z pass
//     maps its plane index through axis_freq as well.
template <int R> struct log2_of { static constexpr int v = R == 1 ? 0 : 1 + log2_of<R / 2>::v; };
template <> struct log2_of<1> { static constexpr int v = 0; };

// Points per lane of the warp transform of a line of L points (S = L / R lanes, S <= 32), and
// whether the line takes the two-pass form (L >= 256, one line per warp) or the single-pass form
// (a lane group of S lanes per line). Up to 128 points, 16 per lane keep most butterflies in
// registers: a 128-point line has 3 lane stages instead of the 5 that 4 per lane would need.
__host__ __device__ constexpr int axis_points_per_lane(int L) {
    return L < 16 ? 4 : (L <= 128 ? 16 : (L == 256 ? 8 : (L == 512 ? 16 : 32)));
}
__host__ __device__ constexpr bool axis_two_pass(int L) { return L >= 256; }
__device__ __forceinline__ int brev_bits(int v, int bits) {
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}
__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }
// Frequency index held at storage position p of a line of L points after the forward transform.
// Single pass (wfft_fwd): p = l + S m holds brev_R(m) + R brev_S(l). Two-pass (wfft2_fwd, S = 32
// lanes in G = 32 / R groups): p = l + 32 c holds brev_R(l / G) + R brev_R(c) + R^2 brev_G(l mod G).
__device__ __forceinline__ int axis_freq(int p, int L) {
    const int R = axis_points_per_lane(L);
    const int lgR = ilog2(R), lgS = ilog2(L) - lgR;
    if (!axis_two_pass(L)) {
        const int m = p >> lgS, l = p & ((1 << lgS) - 1);
        return brev_bits(m, lgR) + (brev_bits(l, lgS) << lgR);
    }
    const int lgG = 5 - lgR;
    const int lp = p & 31, c = p >> 5;
    const int j = lp >> lgG, gg = lp & ((1 << lgG) - 1);
    return brev_bits(j, lgR) + (brev_bits(c, lgR) << lgR) + (brev_bits(gg, lgG) << (2 * lgR));
}

__device__ __forceinline__ double2 shfl_xor_c(double2 v, int m) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ float2 shfl_xor_c(float2 v, int m) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
template <typename C> __device__ __forceinline__ C conj_c(C a) { a.y = -a.y; return a; }

// w_32^t = exp(-2 pi i t / 32), t < 32: the twiddles of the in-register stages (R <= 32), at
// offsets known at compile time, so they are read from the constant bank. Each translation unit
// that includes this header has its own copy; axis_twiddles_init() fills it on the current device.
static __constant__ double2 c_w32d[32];
static __constant__ float2 c_w32f[32];
template <typename C> __device__ __forceinline__ C w32(int t);
template <> __device__ __forceinline__ double2 w32<double2>(int t) { return c_w32d[t]; }
template <> __device__ __forceinline__ float2 w32<float2>(int t) { return c_w32f[t]; }

// d w_32^t and d conj(w_32^t) for a t known at compile time (the unrolled stages): t = 8 is -i,
// a swap and a sign change instead of a complex multiply.
template <typename C> __device__ __forceinline__ C mul_w32(const C &d, int t) {
    if (t == 8) { C r; r.x = d.y; r.y = -d.x; return r; }
    return cmul(d, w32<C>(t));
}
template <typename C> __device__ __forceinline__ C mul_w32c(const C &d, int t) {
    if (t == 8) { C r; r.x = -d.y; r.y = d.x; return r; }
    return cmul(d, conj_c(w32<C>(t)));
}

static inline cudaError_t axis_twiddles_init() {
    double2 d[32];
    float2 f[32];
    for (int t = 0; t < 32; ++t) {
        const long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)t / 32.0L;
        d[t] = make_double2((double)cosl(a), (double)sinl(a));
        f[t] = make_float2((float)cosl(a), (float)sinl(a));
    }
    cudaError_t e = cudaMemcpyToSymbol(c_w32d, d, sizeof(d));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_w32f, f, sizeof(f));
    return e;
}

// Forward lane stage h over the R values of each lane: the lower lane of a pair keeps a + b, the
// upper one (a - b) w. Both are t w~ with t = o + sgn v (sgn = -1 on the upper lane) and w~ = 1 on
// the lower lane, so every lane runs the same instructions (no divergent halves). TW = false for
// h = 1, whose twiddle is w_L^0 = 1 on both lanes. tsh = log2(L / (2 h)) (the twiddle stride).
template <typename C, int R, bool TW>
__device__ __forceinline__ void lane_stage_fwd(C (&v)[R], int l, int h, int tsh, const C *__restrict__ tw) {
    typedef typename real_of<C>::type Rt;
    const bool upper = (l & h) != 0;
    const Rt sg = upper ? (Rt)-1 : (Rt)1;
    C w;
    if (TW) {
        w = tw[(l & (h - 1)) << tsh];
        if (!upper) { w.x = (Rt)1; w.y = (Rt)0; }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const C o = shfl_xor_c(v[m], h);
        C t;
        t.x = fma(sg, v[m].x, o.x);
        t.y = fma(sg, v[m].y, o.y);
        v[m] = TW ? cmul(t, w) : t;
    }
}
// Inverse lane stage h: the upper lane sends u = conj(w) b', the lower one a'; the lower lane keeps
// a' + u, the upper one a' - u, i.e. o + sgn send with sgn = -1 on the upper lane.
template <typename C, int R, bool TW>
__device__ __forceinline__ void lane_stage_inv(C (&v)[R], int l, int h, int tsh, const C *__restrict__ tw) {
    typedef typename real_of<C>::type Rt;
    const bool upper = (l & h) != 0;
    const Rt sg = upper ? (Rt)-1 : (Rt)1;
    C w;
    if (TW) {
        w = conj_c(tw[(l & (h - 1)) << tsh]);
        if (!upper) { w.x = (Rt)1; w.y = (Rt)0; }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const C send = TW ? cmul(v[m], w) : v[m];
        const C o = shfl_xor_c(send, h);
        v[m].x = fma(sg, send.x, o.x);
        v[m].y = fma(sg, send.y, o.y);
    }
}

// Forward transform of one line: v[m] = x[l + S m] on entry, v[m] = X[axis_freq(l + S m)] on
// exit (unnormalised, w_L = exp(-2 pi i / L), tw[j] = w_L^j). Every lane of the warp must call it.
template <typename C, int R>
__device__ __forceinline__ void wfft_fwd(C (&v)[R], int l, int S, int L, const C *__restrict__ tw) {
    constexpr int lgR = log2_of<R>::v;
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const C a = v[b + j], c = v[b + j + h];
                v[b + j] = cadd(a, c);
                const C d = csub(a, c);
                v[b + j + h] = j == 0 ? d : mul_w32(d, j * (16 / h));
            }
        }
    }
#pragma unroll
    for (int m = 1; m < R; ++m) {
        const int k1 = (int)(__brev((unsigned)m) >> (32 - lgR));
        v[m] = cmul(v[m], tw[(l * k1) & (L - 1)]);
    }
    const int lgL = ilog2(L);
    int lgh = ilog2(S) - 1;
    for (int h = S >> 1; h >= 2; h >>= 1, --lgh) lane_stage_fwd<C, R, true>(v, l, h, lgL - 1 - lgh, tw);
    if (S >= 2) lane_stage_fwd<C, R, false>(v, l, 1, 0, tw);
}

// Inverse of wfft_fwd up to the factor L: storage order in, natural order out (unnormalised
// inverse DFT). Every lane of the warp must call it.
template <typename C, int R>
__device__ __forceinline__ void wfft_inv(C (&v)[R], int l, int S, int L, const C *__restrict__ tw) {
    constexpr int lgR = log2_of<R>::v;
    const int lgL = ilog2(L);
    if (S >= 2) lane_stage_inv<C, R, false>(v, l, 1, 0, tw);
    int lgh = 1;
    for (int h = 2; h < S; h <<= 1, ++lgh) lane_stage_inv<C, R, true>(v, l, h, lgL - 1 - lgh, tw);
#pragma unroll
    for (int m = 1; m < R; ++m) {
        const int k1 = (int)(__brev((unsigned)m) >> (32 - lgR));
        v[m] = cmul(v[m], conj_c(tw[(l * k1) & (L - 1)]));
    }
#pragma unroll
    for (int h = 1; h < R; h <<= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const C t = j == 0 ? v[b + j + h] : mul_w32c(v[b + j + h], j * (16 / h));
                const C a = v[b + j];
                v[b + j] = cadd(a, t);
                v[b + j + h] = csub(a, t);
            }
        }
    }
}

// In-register radix-2 stages over R values (compile-time twiddles w_{2h}^j = w_32^(16 j / h)).
template <typename C, int R> __device__ __forceinline__ void regs_dif(C (&v)[R]) {
#pragma unroll
    for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const C a = v[b + j], c = v[b + j + h];
                v[b + j] = cadd(a, c);
                const C d = csub(a, c);
                v[b + j + h] = j == 0 ? d : mul_w32(d, j * (16 / h));
            }
        }
    }
}
template <typename C, int R> __device__ __forceinline__ void regs_dit(C (&v)[R]) {
#pragma unroll
    for (int h = 1; h < R; h <<= 1) {
#pragma unroll
        for (int b = 0; b < R; b += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const C t = j == 0 ? v[b + j + h] : mul_w32c(v[b + j + h], j * (16 / h));
                const C a = v[b + j];
                v[b + j] = cadd(a, t);
                v[b + j + h] = csub(a, t);
            }
        }
    }
}

// Two-pass warp transform of a line of L = 32 R points (R >= 8), one line per warp: the lane
// dimension (32 points) is split as 32 = G x R (G = 32 / R) so that most butterflies run in
// registers instead of across lanes. Pass A: lane l holds x[l + 32 m]; R-point DFT over m,
// twiddle w_L^(l k1). Transpose through the line's shared memory (rows of 32 + G elements, so
// that the gathers hit distinct banks): lane (j, g) = (l / G, l mod G) takes the R values of
// row j at columns g + G t. Pass B: R-point DFT over t, twiddle w_32^(g c), then log2 G stages
// across the G lanes of a group. The result is in the order of axis_freq; `line` must have room
// for L + 32 elements. Every lane of the warp must call it.
template <typename C, int R>
__device__ __forceinline__ void wfft2_fwd(C (&v)[R], C *line, int l, int L, const C *__restrict__ tw) {
    constexpr int G = 32 / R, lgR = log2_of<R>::v, rs = 32 + G;
    regs_dif<C, R>(v);
#pragma unroll
    for (int m = 1; m < R; ++m) {
        const int k1 = (int)(__brev((unsigned)m) >> (32 - lgR));
        v[m] = cmul(v[m], tw[(l * k1) & (L - 1)]);
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < R; ++m) line[m * rs + l] = v[m];
    __syncwarp();
    const int j = l / G, gg = l & (G - 1);
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = line[j * rs + gg + G * t];
    regs_dif<C, R>(v);
    if (G > 1) {
#pragma unroll
        for (int c = 1; c < R; ++c) {
            const int cc = (int)(__brev((unsigned)c) >> (32 - lgR));
            v[c] = cmul(v[c], tw[(gg * cc * R) & (L - 1)]);
        }
        // lanes of a group differ in their low log2 G bits (gg), so the stages index by l
#pragma unroll
        for (int h = G >> 1; h >= 2; h >>= 1) lane_stage_fwd<C, R, true>(v, l, h, ilog2(L) - 1 - ilog2(h), tw);
        lane_stage_fwd<C, R, false>(v, l, 1, 0, tw);
    }
}
template <typename C, int R>
__device__ __forceinline__ void wfft2_inv(C (&v)[R], C *line, int l, int L, const C *__restrict__ tw) {
    constexpr int G = 32 / R, lgR = log2_of<R>::v, rs = 32 + G;
    const int j = l / G, gg = l & (G - 1);
    if (G > 1) {
        lane_stage_inv<C, R, false>(v, l, 1, 0, tw);
#pragma unroll
        for (int h = 2; h < G; h <<= 1) lane_stage_inv<C, R, true>(v, l, h, ilog2(L) - 1 - ilog2(h), tw);
#pragma unroll
        for (int c = 1; c < R; ++c) {
            const int cc = (int)(__brev((unsigned)c) >> (32 - lgR));
            v[c] = cmul(v[c], conj_c(tw[(gg * cc * R) & (L - 1)]));
        }
    }
    regs_dit<C, R>(v);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < R; ++t) line[j * rs + gg + G * t] = v[t];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = line[m * rs + l];
#pragma unroll
    for (int m = 1; m < R; ++m) {
        const int k1 = (int)(__brev((unsigned)m) >> (32 - lgR));
        v[m] = cmul(v[m], conj_c(tw[(l * k1) & (L - 1)]));
    }
    regs_dit<C, R>(v);
}

// Padding of a shared-memory line (complex elements): with CW columns read per row, the rows of
// one 128-byte phase of a warp access land on distinct banks.
template <typename C> __host__ __device__ constexpr int axis_line_pad(int CW) {
    return (int)(128 / sizeof(C)) / CW;
}
// Stride of a shared-memory line: L plus the padding, plus room for the transposition of the
// two-pass transform where it is used (R >= 8; 32 is a multiple of the bank period, so the
// padding keeps its effect).
template <typename C> __host__ __device__ constexpr int axis_line_stride(int L, int CW) {
    return L + axis_line_pad<C>(CW) + (axis_two_pass(L) ? 32 : 0);
}

// Transform the lines [0, nlines) of the tile, one line per lane group of S lanes, looping over
// groups of lines when there are more lines than warps. INV selects the inverse network.
template <typename C, int R, bool TWO, bool INV>
__device__ __forceinline__ void axis_lines(C *s, int nlines, int LS, int L, const C *__restrict__ tw) {
    const int lgS = ilog2(L) - log2_of<R>::v, S = 1 << lgS;
    const int lpw = 32 >> lgS;  // lines per warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int l = lane & (S - 1);
    for (int grp = warp; grp * lpw < nlines; grp += nwarps) {  // uniform across the warp
        const int line = grp * lpw + (lane >> lgS);
        const bool valid = line < nlines;
        C *p = s + (size_t)(valid ? line : 0) * LS;
        C v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = p[l + S * m];
        if constexpr (TWO) {  // S = 32: one line per warp, every lane of it valid or not
            if constexpr (INV) wfft2_inv<C, R>(v, p, l, L, tw);
            else wfft2_fwd<C, R>(v, p, l, L, tw);
        } else {
            if constexpr (INV) wfft_inv<C, R>(v, l, S, L, tw);
            else wfft_fwd<C, R>(v, l, S, L, tw);
        }
        __syncwarp();
        if (valid) {
#pragma unroll
            for (int m = 0; m < R; ++m) p[l + S * m] = v[m];
        }
        __syncwarp();
    }
}

// Threads per CTA at most: 512, or 256 where a lane holds 16 or more values (more registers each).
template <typename T> __host__ __device__ constexpr int axis_max_threads(int R) {
    return (R >= 16 || (sizeof(T) == 8 && R >= 8)) ? 256 : 512;
}
// Dispatch key of the column-pass instances: points per lane and form.
enum { AXK_4 = 0, AXK_16 = 1, AXK_8T = 2, AXK_16T = 3, AXK_32T = 4 };
__host__ __device__ constexpr int axis_form(int L) {
    return axis_two_pass(L) ? (L == 256 ? AXK_8T : (L == 512 ? AXK_16T : AXK_32T)) : (L < 16 ? AXK_4 : AXK_16);
}
template <int K> struct axis_form_of {
    static constexpr int R = K == AXK_4 ? 4 : (K == AXK_8T ? 8 : (K == AXK_32T ? 32 : 16));
    static constexpr bool TWO = K >= AXK_8T;
};

template <typename T, int NCI, int NCO, int MODE, int K, class Op>
__device__ __forceinline__ void axis_body(const Geom &g, int axis, int CW,
                                          const typename cplx_of<T>::type *__restrict__ spec_in,
                                          typename cplx_of<T>::type *spec_out, const Op &op,
                                          const typename cplx_of<T>::type *__restrict__ tw, Scal *sc) {
    typedef typename cplx_of<T>::type C;
    constexpr int NOUT = (MODE == AX_FWD_OP_INV) ? NCO : NCI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    if (op.skip_if_done && sc->done) return;
    const int L = axis == 1 ? g.ny : g.nz;
    const int lgL = axis == 1 ? g.ly : g.lz;
    const int lgCW = ilog2(CW);
    const int LS = axis_line_stride<C>(L, CW);
    const int kx0 = blockIdx.x * CW;
    const int other = blockIdx.y;
    // element offsets in 32 bits: every spectrum of a valid configuration (at most 2^24 voxels,
    // x padded to Px <= max(16, nx/2 + 16)) has fewer than 2^29 elements over all its components
    const unsigned Nh = (unsigned)g.Nh;
    const unsigned lstride = axis == 1 ? (unsigned)g.Px : (unsigned)g.Px * g.ny;
    const unsigned base = (axis == 1 ? (unsigned)other * g.ny * g.Px : (unsigned)other * g.Px) + kx0;
    const int nth = blockDim.x;
    const int npt = L * CW;  // points of one component in the tile
    // 1. coalesced load: i = (c, pos, cc), cc fastest. Each thread issues UB loads before it
    //    stores any of them, so that many loads are in flight. The tile belongs to this CTA alone
    //    and is read before any of it is written back, so the read-only path is safe in place.
    //    (Asynchronous 8-byte copies straight to shared memory measured 1.3-2x slower.)
    constexpr int UB = 8;
    for (int i0 = threadIdx.x; i0 < NCI * npt; i0 += nth * UB) {
        C tmp[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int i = i0 + u * nth;
            if (i < NCI * npt) {
                const int c = i >> (lgL + lgCW);
                const int rem = i & (npt - 1);
                const int pos = rem >> lgCW, cc = rem & (CW - 1);
                tmp[u] = __ldg(spec_in + (c * Nh + base + pos * lstride + cc));
            }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int i = i0 + u * nth;
            if (i < NCI * npt) {
                const int c = i >> (lgL + lgCW);
                const int rem = i & (npt - 1);
                const int pos = rem >> lgCW, cc = rem & (CW - 1);
                s[((c << lgCW) + cc) * LS + pos] = tmp[u];
            }
        }
    }
    __syncthreads();
    // 2. transforms (and the operator between them)
    constexpr int R = axis_form_of<K>::R;
    constexpr bool TWO = axis_form_of<K>::TWO;
    axis_lines<C, R, TWO, MODE == AX_INV>(s, NCI * CW, LS, L, tw);
    if constexpr (MODE == AX_FWD_OP_INV) {
        __syncthreads();
        for (int i = threadIdx.x; i < npt; i += nth) {
            const int cc = i >> lgL, p = i & (L - 1);
            const int kk = axis_freq(p, L);
            const int kx = kx0 + cc;
            const int ky = axis == 1 ? kk : axis_freq(other, g.ny);
            const int kz = axis == 1 ? (g.nz > 1 ? other : 0) : kk;
            C in[NCI], out[NCO];
#pragma unroll
            for (int c = 0; c < NCI; ++c) in[c] = s[((c << lgCW) + cc) * LS + p];
            op.apply(g, kx, ky, kz, in, out);
#pragma unroll
            for (int c = 0; c < NCO; ++c) s[((c << lgCW) + cc) * LS + p] = out[c];
        }
        __syncthreads();
        axis_lines<C, R, TWO, true>(s, NCO * CW, LS, L, tw);
    }
    __syncthreads();
    // 3. coalesced store
    for (int i = threadIdx.x; i < NOUT * npt; i += nth) {
        const int c = i >> (lgL + lgCW);
        const int rem = i & (npt - 1);
        const int pos = rem >> lgCW, cc = rem & (CW - 1);
        spec_out[c * Nh + base + pos * lstride + cc] = s[((c << lgCW) + cc) * LS + pos];
    }
}

template <typename T, int NCI, int NCO, int MODE, int K, class Op>
__global__ void __launch_bounds__(axis_max_threads<T>(axis_form_of<K>::R))
    k_axis(Geom g, int axis, int CW, const typename cplx_of<T>::type *__restrict__ spec_in,
           typename cplx_of<T>::type *spec_out, Op op, const typename cplx_of<T>::type *__restrict__ tw, Scal *sc) {
    axis_body<T, NCI, NCO, MODE, K>(g, axis, CW, spec_in, spec_out, op, tw, sc);
}

template <typename T, int NCI, int NCO, int MODE, int K, class Op>
__global__ void __launch_bounds__(axis_max_threads<T>(axis_form_of<K>::R))
    k_axis_b(Geom g, int axis, int CW, SlotArgs<Op> args, const typename cplx_of<T>::type *__restrict__ tw) {
    typedef typename cplx_of<T>::type C;
    const SlotArg<Op> &a = args.a[blockIdx.z];
    axis_body<T, NCI, NCO, MODE, K>(g, axis, CW, (const C *)a.spec, (C *)a.spec, a.f, tw, a.sc);
}


// Launch shape of k_axis for an axis of L points, NM components and CW columns per CTA: one lane
// group of S = L / R lanes per line, at most 16 warps (the warps loop over the lines beyond), and
// the padded lines in dynamic shared memory.
template <typename C> inline void axis_shape(int L, int NM, int CW, int &threads, size_t &smem, int wcap = 16) {
    const int R = axis_points_per_lane(L), S = L / R;
    const long long lanes = (long long)NM * CW * S;
    long long w = (lanes + 31) / 32;
    int wmax = axis_max_threads<typename real_of<C>::type>(R) / 32;
    if (wcap >= 1 && wcap < wmax) wmax = wcap;
    if (w > wmax) w = wmax;
    if (w < 1) w = 1;
    threads = (int)(32 * w);
    smem = (size_t)NM * CW * (size_t)axis_line_stride<C>(L, CW) * sizeof(C);
}

template <typename T, class Op>
using axis_kernel_t = void (*)(Geom, int, int, const typename cplx_of<T>::type *__restrict__, typename cplx_of<T>::type *,
                               Op, const typename cplx_of<T>::type *__restrict__, Scal *);

// The instance of k_axis for the points per lane of an axis of L points.
template <typename T, int NCI, int NCO, int MODE, class Op> inline axis_kernel_t<T, Op> axis_kernel(int L) {
    switch (axis_form(L)) {
    case AXK_4: return k_axis<T, NCI, NCO, MODE, AXK_4, Op>;
    case AXK_16: return k_axis<T, NCI, NCO, MODE, AXK_16, Op>;
    case AXK_8T: return k_axis<T, NCI, NCO, MODE, AXK_8T, Op>;
    case AXK_16T: return k_axis<T, NCI, NCO, MODE, AXK_16T, Op>;
    default: return k_axis<T, NCI, NCO, MODE, AXK_32T, Op>;
    }
}

template <typename T, class Op>
using axis_kernel_b_t = void (*)(Geom, int, int, SlotArgs<Op>, const typename cplx_of<T>::type *__restrict__);
template <typename T, int NCI, int NCO, int MODE, class Op> inline axis_kernel_b_t<T, Op> axis_kernel_b(int L) {
    switch (axis_form(L)) {
    case AXK_4: return k_axis_b<T, NCI, NCO, MODE, AXK_4, Op>;
    case AXK_16: return k_axis_b<T, NCI, NCO, MODE, AXK_16, Op>;
    case AXK_8T: return k_axis_b<T, NCI, NCO, MODE, AXK_8T, Op>;
    case AXK_16T: return k_axis_b<T, NCI, NCO, MODE, AXK_16T, Op>;
    default: return k_axis_b<T, NCI, NCO, MODE, AXK_32T, Op>;
    }
}

// ---- pointwise kernel with deterministic reductions ---------------------------------------------
template <class F>
__global__ void __launch_bounds__(256) k_pointwise_b(long long N, SlotArgs<F> args) {
    const SlotArg<F> &a = args.a[blockIdx.z];
    const F &f = a.f;
    Scal *sc = a.sc;
    if (f.skip_if_done && sc->done) return;
    double acc[F::NR > 0 ? F::NR : 1];
#pragma unroll
    for (int k = 0; k < (F::NR > 0 ? F::NR : 1); ++k) acc[k] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += stride) f.apply(v, acc);
    if constexpr (F::NR > 0) reduce_finalize<F::NR>(acc, a.partials, sc, f.fin(sc), F::MAXRED);
}

template <class F>
__global__ void __launch_bounds__(256) k_pointwise(long long N, F f, double *partials, Scal *sc) {
    if (f.skip_if_done && sc->done) return;
    double acc[F::NR > 0 ? F::NR : 1];
#pragma unroll
    for (int k = 0; k < (F::NR > 0 ? F::NR : 1); ++k) acc[k] = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += stride) f.apply(v, acc);
    if constexpr (F::NR > 0) reduce_finalize<F::NR>(acc, partials, sc, f.fin(sc), F::MAXRED);
}

}  // namespace pff
