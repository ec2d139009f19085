// Explicit instantiation of the row passes for the double-word kernels (the fused FP64
// exec), rank bound 16.
#define NUFFT_INST_T dfloat
#define NUFFT_INST_KM 16
#include "inst_rows.inc"
