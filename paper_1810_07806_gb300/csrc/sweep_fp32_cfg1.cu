// sweep_fp32_cfg1.cu -- FP32 sweeps in tile configuration 1.
#define SWEEP_CFG 1
#include "sweep_fp32.cu"
