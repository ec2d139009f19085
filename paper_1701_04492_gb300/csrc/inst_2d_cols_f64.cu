// Explicit instantiation of the 2D column pass (section 4), FP64.
#include "passes.cuh"

namespace nufft {
template int launch_cols_2d<double>(nufft_plan, const PassArgs<double> &, cudaStream_t);
}
