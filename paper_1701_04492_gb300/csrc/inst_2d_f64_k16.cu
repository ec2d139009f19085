// Explicit instantiation of the 2D row passes (section 4), forward and adjoint, for
// double and rank bound 16.
#include "passes.cuh"

namespace nufft {
template int launch_rows_2d<double, 16>(nufft_plan, const PassArgs<double> &, cudaStream_t);
template int launch_rows_2d_adj<double, 16>(nufft_plan, const PassArgs<double> &, cudaStream_t);
}
