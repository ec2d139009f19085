// Explicit instantiation of the row passes for the double-word kernels (the fused FP64
// exec), rank bound 4.
#define NUFFT_INST_T dfloat
#define NUFFT_INST_KM 4
#include "inst_rows.inc"
