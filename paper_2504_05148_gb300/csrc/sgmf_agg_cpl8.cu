// sgmf_agg_cpl8.cu -- aggregation kernels with 8 disparity cells per lane (Dp = 128).
#include "sgmf_sweep.cuh"

SGMF_AGG_INSTANTIATE(8)
