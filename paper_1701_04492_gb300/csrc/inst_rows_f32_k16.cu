#define NUFFT_INST_T float
#define NUFFT_INST_KM 16
#include "inst_rows.inc"
