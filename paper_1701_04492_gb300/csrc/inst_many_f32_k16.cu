#define NUFFT_INST_KM 16
#include "inst_many.inc"
