// fill.cuh -- deterministic non-zero test data for the autotuners' timing runs.
//
// Timing on zeroed buffers would mislead: GB300 compresses global-memory data, so
// all-zero intermediates move far fewer DRAM bytes than real transforms do.  Values are
// a 32-bit integer hash of the index mapped to [-1, 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nufft {

template <typename R>
__global__ void k_fill_hash(R *__restrict__ v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)i * 2654435761u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        v[i] = (R)((double)h * (1.0 / 2147483648.0) - 1.0);
    }
}

// Bytes written before each timed run to evict the 126 MB L2, so that candidates are
// timed with cold caches as a stream of different inputs would see them.
constexpr size_t L2_FLUSH_BYTES = (size_t)256 << 20;

// n_real real values of type R (a complex buffer of m values: n_real = 2 m).
template <typename R>
inline cudaError_t fill_hash(void *v, int64_t n_real, cudaStream_t s) {
    if (n_real <= 0) return cudaSuccess;
    const int64_t blocks = (n_real + 255) / 256;
    k_fill_hash<R><<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>((R *)v, n_real);
    return cudaGetLastError();
}

}  // namespace nufft
