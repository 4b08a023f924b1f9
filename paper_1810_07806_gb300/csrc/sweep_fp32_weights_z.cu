#define SWEEP_WT 3   // W_Z
#include "sweep_fp32_weights.cu"
