// hooks.cu -- failure injection for tests, and the device allocation wrapper.
//
// Failures are made on the host or by a bounded device wait, never by a fault: an
// injected allocation failure makes the n-th device allocation report
// cudaErrorMemoryAllocation (the caller then unwinds as for a real one), and the wait
// test waits on an mbarrier that nothing completes until its time limit, so that the
// kernel records the timeout and returns with the context intact.
#include <cuda_runtime.h>

#include <atomic>

#include "async_copy.cuh"
#include "nufft_internal.h"

namespace nufft {
namespace {

std::atomic<int> g_fail_after{-1};   // allocations to let through before one fails; -1: off

__global__ void k_wait_nothing(int *err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int cta_failed;
    if (threadIdx.x == 0) {
        cta_failed = 0;
        mbar_init(&bar, 1);   // one arrival expected; none comes
        fence_mbar_init();
    }
    __syncthreads();
    mbar_wait_bounded(&bar, 0, err, &cta_failed);
}

}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
    int n = g_fail_after.load();
    while (n >= 0) {
        if (g_fail_after.compare_exchange_weak(n, n - 1)) {
            if (n == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

}  // namespace nufft

extern "C" int nufft_test_fail_alloc(int after) {
    nufft::g_fail_after.store(after < 0 ? -1 : after);
    return NUFFT_OK;
}

extern "C" int nufft_test_wait_timeout(void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    int *err = nullptr;
    NUFFT_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    int h = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        nufft::k_wait_nothing<<<1, 32, 0, s>>>(err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return NUFFT_ECUDA;
    }
    return h ? NUFFT_ETIMEOUT : NUFFT_OK;
}
