// Explicit instantiation of the 2D row pass (section 4) for FP64 and rank bound 16.
#include "passes.cuh"

namespace nufft {
template int launch_rows_2d<double, 16>(nufft_plan, const PassArgs<double> &, cudaStream_t);
}
