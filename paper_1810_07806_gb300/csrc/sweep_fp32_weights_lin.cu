#define SWEEP_WT 2   // W_LINEAR
#include "sweep_fp32_weights.cu"
