#define NUFFT_INST_KM 12
#include "inst_many.inc"
