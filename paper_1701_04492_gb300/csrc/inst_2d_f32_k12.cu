// Explicit instantiation of the 2D row passes (section 4), forward and adjoint, for
// float and rank bound 12.
#include "passes.cuh"

namespace nufft {
template int launch_rows_2d<float, 12>(nufft_plan, const PassArgs<float> &, cudaStream_t);
template int launch_rows_2d_adj<float, 12>(nufft_plan, const PassArgs<float> &, cudaStream_t);
}
