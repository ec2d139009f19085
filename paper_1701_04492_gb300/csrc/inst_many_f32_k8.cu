#define NUFFT_INST_KM 8
#include "inst_many.inc"
