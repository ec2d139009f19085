#define NUFFT_INST_T double
#define NUFFT_INST_KM 8
#include "inst_rows.inc"
