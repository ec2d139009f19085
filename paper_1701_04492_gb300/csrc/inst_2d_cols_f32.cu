// Explicit instantiation of the 2D column pass (section 4), FP32.
#include "passes.cuh"

namespace nufft {
template int launch_cols_2d<float>(nufft_plan, const PassArgs<float> &, cudaStream_t);
}
