#define NUFFT_INST_T float
#define NUFFT_INST_KM 12
#include "inst_rows.inc"
