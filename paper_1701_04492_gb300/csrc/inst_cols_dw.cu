// Explicit instantiation of the column-pass launchers (pass 1 and pass B) for the
// double-word kernels (the fused FP64 exec).
#include "passes.cuh"

namespace nufft {
template int launch_cols<dfloat>(nufft_plan, const PassArgs<dfloat> &, bool, cudaStream_t);
}
