// Explicit instantiation of the 2D row passes (section 4), forward and adjoint, for
// float and rank bound 8.
#include "passes.cuh"

namespace nufft {
template int launch_rows_2d<float, 8>(nufft_plan, const PassArgs<float> &, cudaStream_t);
template int launch_rows_2d_adj<float, 8>(nufft_plan, const PassArgs<float> &, cudaStream_t);
}
