// FP64 fused multiply-add throughput of the device the library runs on.
//
// The FP64 path of the solver is bounded by min(HBM bandwidth, FP64 arithmetic), and the FP64
// rate of this part is far below its tensor-core rates, so the benchmark measures it instead of
// assuming a datasheet figure: every thread runs kChains independent dependency chains of
// a = a * b + c in double precision, so that the FMA pipe, not the latency of one chain, limits
// the rate. The chains' results are folded into a device sink so that no work is eliminated.
#include <cuda_runtime.h>

#include "../../include/pff_rve.h"

namespace pffpeak {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
static __device__ double g_sink;

__global__ void __launch_bounds__(256) k_dfma(int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 12345.678) g_sink = s;  // never true for these inputs; keeps the chains live
}

}  // namespace pffpeak

extern "C" int rve_fp64_fma_rate(int iters, double *tflops, double *ms_out, void *stream) {
    using namespace pffpeak;
    if (!tflops || iters < 1) return RVE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RVE_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RVE_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return RVE_ECUDA;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return RVE_ECUDA; }
    // warm-up launch, then the timed one
    k_dfma<<<blocks, threads, 0, st>>>(iters / 8 + 1, 0.999999, 1e-7);
    cudaEventRecord(a, st);
    k_dfma<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7);
    cudaEventRecord(b, st);
    int rc = RVE_OK;
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || !(ms > 0.f))
        rc = RVE_ECUDA;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    const double flops = 2.0 * kChains * kUnroll * (double)iters * (double)threads * (double)blocks;
    *tflops = flops / ((double)ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return RVE_OK;
}
