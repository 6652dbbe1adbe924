// sgmf_agg_cpl12.cu -- aggregation kernels with 12 disparity cells per lane (Dp = 192).
#include "sgmf_sweep.cuh"

SGMF_AGG_INSTANTIATE(12)
