// The persistent batch kernel, adjoint direction (pass A and pass B items); see persist.cuh.
#include "persist_kernel.cuh"

namespace nufft {
int launch_persistent_adj(const PState &st, int grid, size_t smem, const ManyIO &io, cudaStream_t s) {
    return launch_persistent_dir<1>(st, grid, smem, io, s);
}
int persistent_blocks_adj(size_t smem, int *out) { return blocks_per_sm_dir<1>(smem, out); }

int launch_persistent(int dir, const PState &st, int grid, size_t smem, const ManyIO &io, cudaStream_t s) {
    return dir == 0 ? launch_persistent_fwd(st, grid, smem, io, s) : launch_persistent_adj(st, grid, smem, io, s);
}
int persistent_blocks_per_sm(int dir, size_t smem, int *out) {
    return dir == 0 ? persistent_blocks_fwd(smem, out) : persistent_blocks_adj(smem, out);
}
}  // namespace nufft
