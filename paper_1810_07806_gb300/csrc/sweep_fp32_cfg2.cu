// sweep_fp32_cfg2.cu -- FP32 sweeps in tile configuration 2.
#define SWEEP_CFG 2
#include "sweep_fp32.cu"
