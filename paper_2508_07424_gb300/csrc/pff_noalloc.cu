// Allocation-free evaluation of the dissipation functional D(phi) and crack surface Gamma(phi).
//
// Some callers cannot allocate device memory at the moment they need this value: code running
// inside a host framework that owns the whole device memory through its own pool, code that
// must not trigger the implicit device synchronisation of cudaMalloc/cudaFree in a latency-
// critical loop, or embedded callers with a fixed memory budget reserved up front. For them this
// file provides rve_dissipation_noalloc: the caller passes device inputs and a device output,
// and every intermediate (half spectra, reduction partials, solver scalars, FFT twiddles) lives
// in one file-scope __device__ array of fixed size that each GPU loading the library holds
// until the process exits.
//
// The computation is the same three fused passes the engine uses for D and Gamma:
// the forward r2c FFT of phi, the spectral gradient i xi~ phi^ (frequency tables built in the
// scratch array), and the inverse c2r FFT with
// the reduction of sum Gc (phi^2/(2l) + l/2 grad phi . A grad phi).
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>

#include "../../include/pff_rve.h"
#include "pff_common.cuh"
#include "pff_functors.cuh"
#include "pff_kernels.cuh"

using namespace pff;

namespace pffnoalloc {

// 8 MiB of scratch: enough for 2D grids up to 512 x 512 and 3D grids up to 32^3, or any other
// shape whose layout (scalars, partial sums, twiddles, half spectra; computed per call) fits.
constexpr size_t kScratchBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices] = {nullptr};

static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
    size_t scal, partials, tw, xi, spec, total;
};

static int cw_of(int L) {
    const int TL = L / 4;
    int cw = 256 / (TL > 0 ? TL : 1);
    if (cw > 16) cw = 16;
    if (cw < 2) cw = 2;
    return cw;
}

// Frequencies xi~ = 2 pi k / n (FFT order, Nyquist set to zero) on one axis; the x axis covers
// the padded half-spectrum columns, whose padding gets zero.
__global__ void k_xi(double *xi, int n, int len, int half) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    const int lim = half ? n / 2 + 1 : n;
    double v = 0.0;
    if (k < lim && 2 * k != n) {
        const int kk = k <= n / 2 ? k : k - n;
        v = 6.283185307179586476925286766559 * (double)kk / (double)n;
    }
    xi[k] = v;
}

__global__ void k_twiddles(double2 *tw, int L) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)L, &s, &c);
    tw[m] = make_double2(c, s);
}

// Epilogue of the last pass: the dissipation density of Eq. (CrackLenght_ani) summed with and
// without Gc, as the engine's, but with the grain ids checked against n_grains before they index
// the caller's tables. The ids come from caller memory that this entry point cannot validate on
// the host, so an id outside [0, n_grains) reads no table entry and turns both sums into NaN.
template <int D>
struct EpiDissChecked {
    static constexpr int NR = 2;
    bool skip_if_done;
    const double *phi;
    const double *GcTab, *Atab;
    const int *gid;
    int n_grains;
    double ell;
    __device__ void apply(long long v, const double *gr, double *acc) const {
        const int gg = gid[v];
        if (gg < 0 || gg >= n_grains) {
            const double nan = __longlong_as_double(0x7ff8000000000000LL);
            acc[0] += nan;
            acc[1] += nan;
            return;
        }
        const double *A = Atab + (size_t)gg * 6;
        double q;
        if constexpr (D == 2) {
            q = gr[0] * (A[0] * gr[0] + A[2] * gr[1]) + gr[1] * (A[2] * gr[0] + A[1] * gr[1]);
        } else {
            q = gr[0] * (A[0] * gr[0] + A[5] * gr[1] + A[4] * gr[2]) +
                gr[1] * (A[5] * gr[0] + A[1] * gr[1] + A[3] * gr[2]) +
                gr[2] * (A[4] * gr[0] + A[3] * gr[1] + A[2] * gr[2]);
        }
        const double p = phi[v];
        const double dens = p * p / (2.0 * ell) + 0.5 * ell * q;
        acc[0] += GcTab[gg] * dens;
        acc[1] += dens;
    }
    struct Fin {
        Scal *sc;
        __device__ void operator()(const double *t) const { sc->D = t[0]; sc->Gamma = t[1]; }
    };
    __device__ Fin fin(Scal *sc) const { return Fin{sc}; }
};

}  // namespace pffnoalloc

using namespace pffnoalloc;

extern "C" int rve_dissipation_noalloc(int dim, const int n[3], double ell, int n_grains, const int32_t *grain_id,
                                       const double *Gc, const double *A, const double *phi, double *out,
                                       void *stream) {
    if (!n || !grain_id || !Gc || !A || !phi || !out || n_grains <= 0 || !(ell > 0)) return RVE_EINVAL;
    if (dim != 2 && dim != 3) return RVE_EINVAL;
    auto pow2 = [](int v) { return v >= 4 && v <= 1024 && (v & (v - 1)) == 0; };
    const int nx = n[0], ny = n[1], nz = dim == 2 ? 1 : n[2];
    // 3D plates one voxel thick (nz = 1) are accepted as by rve_create: no z transform
    if (!pow2(nx) || !pow2(ny) || (dim == 2 ? n[2] != 1 : (nz != 1 && !pow2(nz)))) return RVE_EINVAL;

    Geom g{};
    g.d = dim; g.ns = dim == 2 ? 3 : 6;
    g.nx = nx; g.ny = ny; g.nz = nz;
    auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return l; };
    g.lx = lg(nx); g.ly = lg(ny); g.lz = lg(nz);
    const int cwy = cw_of(ny), cwz = nz > 1 ? cw_of(nz) : 2, cw = cwy > cwz ? cwy : cwz;
    g.Px = ((nx / 2 + 1 + cw - 1) / cw) * cw;
    g.N = (long long)nx * ny * nz;
    g.Nh = (long long)g.Px * ny * nz;
    g.invN = 1.0 / (double)g.N;

    // launch shape of the x passes (same rule as the engine)
    const int TL = nx / 4;
    const long long pairs = (long long)ny * nz / 2;
    int RP = 128 / TL;
    if (RP < 1) RP = 1;
    if (RP > pairs) RP = (int)pairs;
    const int xthreads = RP * TL;
    const int xblocks = (int)(pairs / RP);
    if (xthreads < 32) return RVE_EINVAL;  // the x passes reduce with full-warp shuffles

    // scratch layout; reject grids whose requirement exceeds the static array
    Layout lay;
    lay.scal = 0;
    lay.partials = align256(sizeof(Scal));
    lay.tw = lay.partials + align256(sizeof(double) * 2 * (size_t)xblocks);
    lay.xi = lay.tw + align256(sizeof(double2) * (size_t)(nx + ny + nz));
    lay.spec = lay.xi + align256(sizeof(double) * (size_t)(g.Px + ny + nz));
    lay.total = lay.spec + align256(sizeof(double2) * (size_t)dim * (size_t)g.Nh);
    if (lay.total > kScratchBytes) {
        std::fprintf(stderr,
                     "rve_dissipation_noalloc: grid %dx%dx%d needs %zu bytes of scratch, more than the fixed %zu\n",
                     nx, ny, nz, lay.total, kScratchBytes);
        return RVE_EINVAL;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RVE_ECUDA;
    if (!g_scratch_addr[dev]) {
        // one-time set-up on this device (the device is current): the host-side name of
        // g_scratch is not a device address, so look the address up and keep it.
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RVE_ECUDA;
        // the column passes read their in-register twiddles from this file's constant bank
        if (axis_twiddles_init() != cudaSuccess) return RVE_ECUDA;
        g_scratch_addr[dev] = p;
    }
    unsigned char *base = (unsigned char *)g_scratch_addr[dev];
    Scal *sc = (Scal *)(base + lay.scal);
    double *partials = (double *)(base + lay.partials);
    double2 *twx = (double2 *)(base + lay.tw);
    double2 *twy = twx + nx;
    double2 *twz = twy + ny;
    double *xix = (double *)(base + lay.xi);
    double *xiy = xix + g.Px;
    double *xiz = xiy + ny;
    const XiTab<double> xi{xix, xiy, xiz};
    double2 *spec = (double2 *)(base + lay.spec);
    cudaStream_t st = (cudaStream_t)stream;

    // state left by an earlier call is not trusted: reset the scalars (the reduction counter
    // must start at zero) and the spectral buffer (its padding columns are read by the FFTs).
    if (cudaMemsetAsync(sc, 0, sizeof(Scal), st) != cudaSuccess) return RVE_ECUDA;
    if (cudaMemsetAsync(spec, 0, sizeof(double2) * (size_t)dim * (size_t)g.Nh, st) != cudaSuccess) return RVE_ECUDA;
    k_twiddles<<<(nx + 255) / 256, 256, 0, st>>>(twx, nx);
    k_twiddles<<<(ny + 255) / 256, 256, 0, st>>>(twy, ny);
    if (nz > 1) k_twiddles<<<(nz + 255) / 256, 256, 0, st>>>(twz, nz);
    k_xi<<<(g.Px + 255) / 256, 256, 0, st>>>(xix, nx, g.Px, 1);
    k_xi<<<(ny + 255) / 256, 256, 0, st>>>(xiy, ny, ny, 0);
    k_xi<<<(nz + 255) / 256, 256, 0, st>>>(xiz, nz, nz, 0);

    const size_t smx = (size_t)RP * nx * sizeof(double2);
    auto axis_launch = [&](auto kernel, int ax, int NM, const auto &op, const double2 *tw) -> cudaError_t {
        const int L = ax == 1 ? ny : nz;
        const int CW = ax == 1 ? cwy : cwz;
        int threads;
        size_t sm;
        axis_shape<double2>(L, NM, CW, threads, sm);
        if (sm > 32 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kernel<<<dim3(g.Px / CW, ax == 1 ? nz : ny), threads, sm, st>>>(g, ax, CW, spec, spec, op, tw, sc);
        return cudaGetLastError();
    };

    // forward x pass of phi
    {
        auto k = k_x_fwd<double, 1, ProField<double>>;
        k<<<xblocks, xthreads, smx, st>>>(g, ProField<double>{false, phi}, spec, twx, partials, sc);
        if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    }
    const int32_t *gid = grain_id;
    if (dim == 2) {
        if (axis_launch(axis_kernel<double, 1, 2, AX_FWD_OP_INV, OpGrad<double2, 2>>(ny), 1, 2, OpGrad<double2, 2>{false, xi}, twy))
            return RVE_ECUDA;
        auto k = k_x_inv<double, 2, EpiDissChecked<2>>;
        const size_t sm = smx * 2;
        if (sm > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<xblocks, xthreads, sm, st>>>(g, spec, EpiDissChecked<2>{false, phi, Gc, A, gid, n_grains, ell}, twx,
                                         partials, sc);
    } else {
        if (nz == 1) {
            // plate: xi_z = 0, so the gradient is taken in the y pass, as in 2D
            if (axis_launch(axis_kernel<double, 1, 3, AX_FWD_OP_INV, OpGrad<double2, 3>>(ny), 1, 3, OpGrad<double2, 3>{false, xi},
                            twy))
                return RVE_ECUDA;
        } else {
            if (axis_launch(axis_kernel<double, 1, 1, AX_FWD, OpGrad<double2, 3>>(ny), 1, 1, OpGrad<double2, 3>{false, xi}, twy))
                return RVE_ECUDA;
            if (axis_launch(axis_kernel<double, 1, 3, AX_FWD_OP_INV, OpGrad<double2, 3>>(nz), 2, 3, OpGrad<double2, 3>{false, xi},
                            twz))
                return RVE_ECUDA;
            if (axis_launch(axis_kernel<double, 3, 3, AX_INV, OpGrad<double2, 3>>(ny), 1, 3, OpGrad<double2, 3>{false, xi}, twy))
                return RVE_ECUDA;
        }
        auto k = k_x_inv<double, 3, EpiDissChecked<3>>;
        const size_t sm = smx * 3;
        if (sm > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k<<<xblocks, xthreads, sm, st>>>(g, spec, EpiDissChecked<3>{false, phi, Gc, A, gid, n_grains, ell}, twx,
                                         partials, sc);
    }
    if (cudaGetLastError() != cudaSuccess) return RVE_ECUDA;
    // D and Gamma were written to the scalar block by the last CTA; hand them to the caller.
    if (cudaMemcpyAsync(out, &sc->D, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) return RVE_ECUDA;
    if (cudaMemcpyAsync(out + 1, &sc->Gamma, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RVE_ECUDA;
    return RVE_OK;
}
