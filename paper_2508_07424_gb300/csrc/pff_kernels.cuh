// Fused spectral passes of the FFT phase-field-fracture solver (sm_103a).
//
// A spectral operator  v -> F^-1[ Op(xi) F[ pro(v) ] ]  is applied as
//   k_x_fwd   : per pair of x-rows, evaluate the prologue (e.g. the stress C_phi : p of a CG
//               direction) for NC components, pack the two real rows as one complex line, FFT
//               along x in shared memory, split into the two half spectra, store [c][z][y][kx];
//   k_axis    : per tile of CW adjacent kx columns, FFT along y (2D) or y then z (3D) in shared
//               memory, apply the per-frequency operator (projection, gradient, divergence,
//               preconditioner), inverse FFT, store;
//   k_x_inv   : rebuild the packed line from two half spectra, inverse FFT along x, evaluate the
//               epilogue (CG vector update, residual, dot products) with a deterministic
//               reduction finalised by the last CTA.
//   k_x_mid   : inverse x pass, a pointwise map (damage flux Gc l A grad phi), forward x pass.
// All kernels of one solve read their scalars (alpha, beta, done flag) from a device Scal block,
// so a whole CG iteration is launched without host synchronisation.
#pragma once

#include "pff_common.cuh"

namespace pff {

enum { AX_FWD = 0, AX_INV = 1, AX_FWD_OP_INV = 2 };

// ---- x-axis forward (r2c) pass ------------------------------------------------------------------
template <typename T, int NC, class Pro>
__global__ void __launch_bounds__(512) k_x_fwd(Geom g, Pro pro, typename cplx_of<T>::type *__restrict__ spec,
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
__global__ void __launch_bounds__(512) k_x_inv(Geom g, const typename cplx_of<T>::type *__restrict__ spec, Epi epi,
                                               const typename cplx_of<T>::type *__restrict__ tw, double *partials,
                                               Scal *sc) {
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
    double acc[Epi::NR > 0 ? Epi::NR : 1];
#pragma unroll
    for (int k = 0; k < (Epi::NR > 0 ? Epi::NR : 1); ++k) acc[k] = 0.0;
    const T sN = (T)g.invN;
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
        epi.apply(row0 + x, va, acc);
        epi.apply(row0 + nx + x, vb, acc);
    }
    if constexpr (Epi::NR > 0) reduce_finalize<Epi::NR>(acc, partials, sc, epi.fin(sc));
}

// ---- x-axis inverse, pointwise map, x-axis forward ----------------------------------------------
// Inverse x pass of NCI components, mid.apply(v, in[NCI], out[NCO]) per voxel (NCO <= NCI), forward
// x pass of the NCO outputs.
template <typename T, int NCI, int NCO, class Mid>
__global__ void __launch_bounds__(512) k_x_mid(Geom g, typename cplx_of<T>::type *__restrict__ spec, Mid mid,
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

// ---- y / z axis pass ------------------------------------------------------------------------------
// axis = 1 (y) or 2 (z). A CTA owns CW adjacent kx columns of one plane (z for axis y, y for
// axis z) and all L points along the axis. MODE: AX_FWD, AX_INV or AX_FWD_OP_INV (forward, the
// per-frequency operator mapping NCI -> NCO components, inverse).
template <typename T, int NCI, int NCO, int MODE, class Op>
__global__ void __launch_bounds__(512) k_axis(Geom g, int axis, const typename cplx_of<T>::type *spec_in,
                                              typename cplx_of<T>::type *spec_out, Op op,
                                              const typename cplx_of<T>::type *__restrict__ tw, Scal *sc) {
    typedef typename cplx_of<T>::type C;
    constexpr int NM = NCI > NCO ? NCI : NCO;
    constexpr int NOUT = (MODE == AX_FWD_OP_INV) ? NCO : NCI;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *s = reinterpret_cast<C *>(smem_raw);
    if (op.skip_if_done && sc->done) return;
    const int L = axis == 1 ? g.ny : g.nz;
    const int logL = axis == 1 ? g.ly : g.lz;
    const int TL = L >> 2;
    const int CW = blockDim.x / TL;
    const int kx0 = blockIdx.x * CW;
    const int other = blockIdx.y;
    const long long lstride = axis == 1 ? (long long)g.Px : (long long)g.Px * g.ny;
    const long long base = axis == 1 ? (long long)other * g.ny * g.Px : (long long)other * g.Px;
    // blockDim.x = CW * L / 4: every loop over the tile's L * CW points takes exactly 4 steps,
    // unrolled (fully up to 4 components, by 2 beyond, to stay within the register budget)
    constexpr int UQ = NM <= 4 ? 4 : 2;
    const int nthreads = blockDim.x;
#pragma unroll UQ
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.x + q * nthreads;
        const int pos = i / CW, cc = i - pos * CW;
#pragma unroll
        for (int c = 0; c < NCI; ++c)
            s[(size_t)(c * CW + cc) * L + pos] = spec_in[(size_t)c * g.Nh + base + pos * lstride + kx0 + cc];
    }
    __syncthreads();
    if constexpr (MODE == AX_INV) {
        fft_lines<C, NM>(s, L, logL, NCI, 1, CW, tw, true);
    } else {
        fft_lines<C, NM>(s, L, logL, NCI, 1, CW, tw, false);
    }
    if constexpr (MODE == AX_FWD_OP_INV) {
#pragma unroll UQ
        for (int q = 0; q < 4; ++q) {
            const int i = threadIdx.x + q * nthreads;
            const int pos = i / CW, cc = i - pos * CW;
            const int kx = kx0 + cc;
            const int ky = axis == 1 ? pos : other;
            const int kz = axis == 1 ? (g.nz > 1 ? other : 0) : pos;
            C in[NCI], out[NCO];
#pragma unroll
            for (int c = 0; c < NCI; ++c) in[c] = s[(size_t)(c * CW + cc) * L + pos];
            op.apply(g, kx, ky, kz, in, out);
#pragma unroll
            for (int c = 0; c < NCO; ++c) s[(size_t)(c * CW + cc) * L + pos] = out[c];
        }
        __syncthreads();
        fft_lines<C, NM>(s, L, logL, NCO, 1, CW, tw, true);
    }
#pragma unroll UQ
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.x + q * nthreads;
        const int pos = i / CW, cc = i - pos * CW;
#pragma unroll
        for (int c = 0; c < NOUT; ++c)
            spec_out[(size_t)c * g.Nh + base + pos * lstride + kx0 + cc] = s[(size_t)(c * CW + cc) * L + pos];
    }
}

// ---- pointwise kernel with deterministic reductions ---------------------------------------------
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
