#define NUFFT_INST_KM 4
#include "inst_many.inc"
