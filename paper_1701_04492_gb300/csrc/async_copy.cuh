// async_copy.cuh -- bulk asynchronous copies global -> shared (the TMA engine's
// cp.async.bulk) completed on shared-memory mbarriers, with bounded waits.
//
// A wait gives up after WAIT_LIMIT_NS of %globaltimer, records the failure in a
// device error word (read back by nufft2_check) and returns, so a copy that never
// lands cannot hang the GPU; after one timeout the CTA skips further waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nufft {

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s

// Bits of the device error word (nufft2_check).
constexpr int ERR_TIMEOUT = 1;   // a bounded wait gave up
constexpr int ERR_INDEX = 2;     // an index check failed (NUFFT_CHECK builds)

// The index check of NUFFT_CHECK builds: ok is the in-range condition of an access the
// caller makes only when this returns true.  A failure is recorded in the error word.
// Without NUFFT_CHECK it is true and the condition is discarded.
__device__ __forceinline__ bool idx_ok(bool ok, int *err) {
#ifdef NUFFT_CHECK
    if (!ok && err) atomicOr(err, ERR_INDEX);
    return ok;
#else
    (void)ok;
    (void)err;
    return true;
#endif
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the mbarrier initialisations visible to the async proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned
// shared dst; completes `bytes` transactions on bar.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of bar to complete, at most WAIT_LIMIT_NS.  On timeout
// sets *err and *cta_failed and returns false; once *cta_failed is set it returns
// false at once.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *err,
                                                  volatile int *cta_failed) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!*cta_failed) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            *cta_failed = 1;
            if (err) atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
    return false;
}

}  // namespace nufft
