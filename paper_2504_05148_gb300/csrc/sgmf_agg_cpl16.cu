// sgmf_agg_cpl16.cu -- aggregation kernels with 16 disparity cells per lane (Dp = 256).
#include "sgmf_sweep.cuh"

SGMF_AGG_INSTANTIATE(16)
