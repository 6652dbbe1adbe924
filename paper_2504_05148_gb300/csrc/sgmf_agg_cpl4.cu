// sgmf_agg_cpl4.cu -- aggregation kernels with 4 disparity cells per lane (Dp = 64).
#include "sgmf_sweep.cuh"

SGMF_AGG_INSTANTIATE(4)
