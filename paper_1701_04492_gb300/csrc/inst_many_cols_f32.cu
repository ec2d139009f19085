// Explicit instantiation of the batched column-pass launchers (pass 1 and pass B over
// many problems per launch), FP32.
#include "passes.cuh"

namespace nufft {
template int launch_cols_many<float>(nufft_plan, const PassArgs<float> *, int, int, bool, const ManyIO &,
                                     cudaStream_t);
}
