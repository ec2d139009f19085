// measure.cu -- the FP32 peak that the roofline of the exec kernels is reported against.
//
// The passes are bound by the plain FP32 pipes (the FFT butterflies, the factor
// recurrences), not by HBM, so their roofline denominator is the FP32 FMA rate of the
// device, measured here rather than taken from a datasheet: every thread runs NCH
// independent FMA chains (enough independent instructions per warp to cover the FMA
// latency), with operands the compiler cannot fold, for `iters` rounds of UNROLL steps.
#include <cuda_runtime.h>

#include "nufft_internal.h"

namespace nufft {
namespace {

constexpr int NCH = 16;      // independent FMA chains per thread
constexpr int UNROLL = 8;    // FMA steps per chain per loop round
constexpr int THREADS = 1024;

__device__ float g_sink[32];

__global__ void __launch_bounds__(THREADS) k_fma_peak(int64_t iters, float b, float c) {
    float a[NCH];
#pragma unroll
    for (int i = 0; i < NCH; ++i) a[i] = 1e-3f * (float)threadIdx.x + (float)i;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int i = 0; i < NCH; ++i) a[i] = fmaf(a[i], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < NCH; ++i) s += a[i];
    // a store that never happens for the operands the host passes (|a| stays far below
    // 1e30), but that the compiler must keep, and with it every FMA
    if (s == 1e30f) g_sink[threadIdx.x & 31] = s;
}

}  // namespace
}  // namespace nufft

extern "C" int nufft_fp32_fma_peak(int64_t iters, int blocks_per_sm, void *stream, float *ms_out,
                                   double *flop_out) {
    if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 2 || !ms_out || !flop_out) return NUFFT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    NUFFT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    NUFFT_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        (void)cudaGetLastError();
        return NUFFT_ECUDA;
    }
    int rc = NUFFT_OK;
    // b < 1 and c > 0: every chain converges to c / (1 - b) without overflow or denormals
    if (cudaEventRecord(e0, s) != cudaSuccess) rc = NUFFT_ECUDA;
    if (!rc) nufft::k_fma_peak<<<blocks, nufft::THREADS, 0, s>>>(iters, 0.9999999f, 1e-7f);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = NUFFT_ECUDA;
    if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = NUFFT_ECUDA;
    if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = NUFFT_ECUDA;
    if (!rc && cudaEventElapsedTime(ms_out, e0, e1) != cudaSuccess) rc = NUFFT_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        (void)cudaGetLastError();
        return rc;
    }
    *flop_out = 2.0 * nufft::NCH * nufft::UNROLL * (double)iters * (double)blocks * nufft::THREADS;
    return NUFFT_OK;
}
