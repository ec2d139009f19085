// The persistent batch kernel, forward direction (pass 1 and pass 2 items); see persist.cuh.
#include "persist_kernel.cuh"

namespace nufft {
int launch_persistent_fwd(const PState &st, int grid, size_t smem, const ManyIO &io, cudaStream_t s) {
    return launch_persistent_dir<0>(st, grid, smem, io, s);
}
int persistent_blocks_fwd(size_t smem, int *out) { return blocks_per_sm_dir<0>(smem, out); }
}  // namespace nufft
