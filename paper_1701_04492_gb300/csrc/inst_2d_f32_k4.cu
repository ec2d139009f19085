// Explicit instantiation of the 2D row pass (section 4) for FP32 and rank bound 4.
#include "passes.cuh"

namespace nufft {
template int launch_rows_2d<float, 4>(nufft_plan, const PassArgs<float> &, cudaStream_t);
}
