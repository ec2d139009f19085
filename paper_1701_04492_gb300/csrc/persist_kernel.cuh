// persist_kernel.cuh -- the persistent batch kernel (see persist.cuh), included once per
// direction by persist_fwd.cu and persist_adj.cu so that the two compile in parallel.
#pragma once

#include "persist.cuh"

namespace nufft {

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Order this thread's earlier generic-proxy accesses to global memory before its later
// async-proxy ones (the bulk copies that read what other CTAs wrote).
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait (bounded) until *cnt reaches need; a wait that gives up records a timeout.
__device__ __forceinline__ void wait_count(const int *cnt, int need, int *err) {
    if (ld_acquire_gpu(cnt) >= need) return;
    const unsigned long long t0 = global_ns();
    while (ld_acquire_gpu(cnt) < need) {
        if (global_ns() - t0 > WAIT_LIMIT_NS) {
            if (err) atomicOr(err, ERR_TIMEOUT);
            return;
        }
        __nanosleep(256);
    }
}

// Each pass, size and rank bound is its own (not inlined) function: the kernel is one
// launch, but the compiler allocates registers per body, as for the class launches, and a
// row pass loops over its class's rank bound KM (8, 12 or 16), not over the largest.  The
// body works on a private copy of the item's arguments (sa is in shared memory, and
// reached through a pointer the compiler could not keep its fields in registers across
// the body's stores).
template <int DIR, int P, int KM>
__device__ __noinline__ void run_first(const PassArgs<float> &sa, const float *beta, const PItem &w) {
    const PassArgs<float> a = sa;
    if constexpr (DIR == 0) {
        (void)beta;
        pass1_body<float, P>(a, w.bx, w.by);
    } else {
        passA_body<float, P, KM>(a, BetaShared<float, KM>{beta}, w.bx);
    }
}
template <int DIR, int P, int KM>
__device__ __noinline__ void run_second(const PassArgs<float> &sa, const float *beta, const PItem &w) {
    const PassArgs<float> a = sa;
    if constexpr (DIR == 0) {
        pass2_body<float, P, KM>(a, BetaShared<float, KM>{beta}, w.bx);
    } else {
        (void)beta;
        passB_body<float, P>(a, w.bx, w.by);
    }
}

// the row pass of the item's kind takes the class's rank bound; the column pass none
template <int DIR, int P>
__device__ __forceinline__ void run_sized(const PassArgs<float> &a, const float *beta, const PItem &w, int km) {
    const bool row = (w.kind == 0) == (DIR == 1);
    if (w.kind == 0) {
        if (!row) run_first<DIR, P, 16>(a, beta, w);
        else if (km <= 8) run_first<DIR, P, 8>(a, beta, w);
        else if (km <= 12) run_first<DIR, P, 12>(a, beta, w);
        else run_first<DIR, P, 16>(a, beta, w);
    } else {
        if (!row) run_second<DIR, P, 16>(a, beta, w);
        else if (km <= 8) run_second<DIR, P, 8>(a, beta, w);
        else if (km <= 12) run_second<DIR, P, 12>(a, beta, w);
        else run_second<DIR, P, 16>(a, beta, w);
    }
}

template <int DIR>
__device__ __forceinline__ void run_block(const PassArgs<float> &a, const float *beta, PItem w, int P, int km) {
    switch (P) {
        case 32: run_sized<DIR, 32>(a, beta, w, km); break;
        case 64: run_sized<DIR, 64>(a, beta, w, km); break;
        case 128: run_sized<DIR, 128>(a, beta, w, km); break;
        case 256: run_sized<DIR, 256>(a, beta, w, km); break;
        default: run_sized<DIR, 512>(a, beta, w, km); break;
    }
}

template <int DIR>
__global__ void __launch_bounds__(256, 2) k_persist(const PState st, const ManyIO io) {
    __shared__ PassArgs<float> a;
    __shared__ Beta<float, 16> sb;
    __shared__ int s_item, s_last;
    int next = 0;   // thread 0: the ticket taken for the item after the current one
    if (threadIdx.x == 0) s_item = atomicAdd(&st.ctl[0], 1);
    __syncthreads();
    for (;;) {
        const int it = s_item;
        if (it >= st.n_items) break;
        // the next ticket is in flight while this item runs
        if (threadIdx.x == 0) next = atomicAdd(&st.ctl[0], 1);
        const PItem w = st.items[it];
        const PClass c = st.classes[w.cls];
        // the item's arguments, and its coefficients as a km x km table, to shared memory
        const int km = c.km;
        {
            const unsigned long long *src =
                reinterpret_cast<const unsigned long long *>(c.args[w.kind] + w.member);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(&a);
            for (int i = threadIdx.x; i < (int)(sizeof(PassArgs<float>) / 8); i += blockDim.x) dst[i] = src[i];
            const float *bsrc = &st.betas[w.prob].b[0][0];
            for (int i = threadIdx.x; i < km * km; i += blockDim.x) (&sb.b[0][0])[i] = bsrc[(i / km) * 16 + i % km];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            a.in = (const float2 *)io.in + a.in_off;
            a.out = (float2 *)io.out + a.out_off;
            // a second pass reads what the problem's first pass wrote
            if (w.kind == 1) {
                wait_count(&st.done[w.prob], st.need[w.prob], a.err);
                fence_proxy_async_global();
            }
        }
        __syncthreads();
        const int P = w.kind == 0 ? (DIR == 0 ? c.P_cols : c.P_rows) : (DIR == 0 ? c.P_rows : c.P_cols);
        for (int q = 0; q < w.nbx; ++q) {
            PItem wq = w;
            wq.bx = w.bx + q;
            run_block<DIR>(a, &sb.b[0][0], wq, P, km);
            // the block's mbarriers, quiescent now (every copy was waited for), are
            // invalidated before shared memory is reused
            __syncthreads();
            if (threadIdx.x == 0 && w.kind == 1) {
                if (DIR == 0) {
                    const int gs = a.G > 0 ? a.G : 1;
                    uint64_t *mb = reinterpret_cast<uint64_t *>(
                        reinterpret_cast<unsigned char *>(smem_base<float>()) + a.mbar_off);
                    for (int m = 0; m < gs * a.B2; ++m) mbar_inval(&mb[m]);
                } else {
                    uint64_t *mb = reinterpret_cast<uint64_t *>(smem_base<float>() + 2 * a.C * a.S);
                    mbar_inval(&mb[0]);
                    mbar_inval(&mb[1]);
                }
            }
            __syncthreads();
        }
        // a first-pass item's writes are made visible GPU-wide by every thread before its
        // count is published (the second pass reads them); a second-pass item has no reader
        if (w.kind == 0) {
            __threadfence();
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (w.kind == 0) atomicAdd(&st.done[w.prob], w.nbx);
            s_item = next;
        }
        __syncthreads();
    }
    // the last CTA to leave resets the ticket and the counters for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st.ctl[1], 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        for (int i = threadIdx.x; i < st.nprob; i += blockDim.x) st.done[i] = 0;
        if (threadIdx.x == 0) {
            st.ctl[0] = 0;
            st.ctl[1] = 0;
        }
        __threadfence();
    }
}

template <int DIR>
int launch_persistent_dir(const PState &st, int grid, size_t smem, const ManyIO &io, cudaStream_t s) {
    static SmemFlags done{};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return NUFFT_ECUDA;
    }
    if (int rc = set_smem(k_persist<DIR>, smem, dev, done)) return rc;
    k_persist<DIR><<<grid, 256, smem, s>>>(st, io);
    return launch_status();
}

template <int DIR>
int blocks_per_sm_dir(size_t smem, int *out) {
    int dev = 0;
    static SmemFlags done{};
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return NUFFT_ECUDA;
    }
    if (int rc = set_smem(k_persist<DIR>, smem, dev, done)) return rc;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_persist<DIR>, 256, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return NUFFT_ECUDA;
    }
    return NUFFT_OK;
}

}  // namespace nufft
