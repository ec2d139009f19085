// Explicit instantiation of the 2D column passes (section 4), forward and adjoint, double.
#include "passes.cuh"

namespace nufft {
template int launch_cols_2d<double>(nufft_plan, const PassArgs<double> &, cudaStream_t);
template int launch_cols_2d_adj<double>(nufft_plan, const PassArgs<double> &, cudaStream_t);
}
