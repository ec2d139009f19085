#define NUFFT_INST_T double
#define NUFFT_INST_KM 12
#include "inst_rows.inc"
