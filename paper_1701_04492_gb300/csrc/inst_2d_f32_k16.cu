// Explicit instantiation of the 2D row pass (section 4) for FP32 and rank bound 16.
#include "passes.cuh"

namespace nufft {
template int launch_rows_2d<float, 16>(nufft_plan, const PassArgs<float> &, cudaStream_t);
}
