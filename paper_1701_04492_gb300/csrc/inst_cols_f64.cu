// Explicit instantiation of the column-pass launchers (pass 1 and pass B).
#include "passes.cuh"

namespace nufft {
template int launch_cols<double>(nufft_plan, const PassArgs<double> &, bool, cudaStream_t);
}
