#define NUFFT_INST_T double
#define NUFFT_INST_KM 16
#include "inst_rows.inc"
