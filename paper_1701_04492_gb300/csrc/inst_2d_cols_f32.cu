// Explicit instantiation of the 2D column passes (section 4), forward and adjoint, float.
#include "passes.cuh"

namespace nufft {
template int launch_cols_2d<float>(nufft_plan, const PassArgs<float> &, cudaStream_t);
template int launch_cols_2d_adj<float>(nufft_plan, const PassArgs<float> &, cudaStream_t);
}
