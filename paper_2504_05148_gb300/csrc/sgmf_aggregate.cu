// sgmf_aggregate.cu -- picks the aggregation kernels for a context's lane
// width (Dp = 16 * CPL cells per line) and path-cost spill width.  The kernel
// templates are in sgmf_aggregate.cuh; each lane width is instantiated in its
// own translation unit (sgmf_agg_cpl*.cu).
#include <cstdint>

#include "sgmf_internal.cuh"

namespace sgmf {

template <int CPL, bool S8>
cudaError_t launch_lines_t(const KParams &k, const Buffers &b, int nf, cudaStream_t s);
template <int CPL, bool S8>
cudaError_t launch_rows_t(const KParams &k, const Buffers &b, int nf, cudaStream_t s);
template <int CPL>
cudaError_t launch_sweep_t(const KParams &k, const Buffers &b, int nf, cudaStream_t s);
template <int CPL>
int sweep_plan_t(const KParams &k, int nb, int *slots);

// Dp = 32 * DPL = 16 * CPL
#define SGMF_DISPATCH(FN, ...)                    \
  switch (k.DPL * 4 + (spill8 ? 1 : 0)) {         \
    case 8: return FN<4, false>(__VA_ARGS__);     \
    case 9: return FN<4, true>(__VA_ARGS__);      \
    case 16: return FN<8, false>(__VA_ARGS__);    \
    case 17: return FN<8, true>(__VA_ARGS__);     \
    case 24: return FN<12, false>(__VA_ARGS__);   \
    case 25: return FN<12, true>(__VA_ARGS__);    \
    case 32: return FN<16, false>(__VA_ARGS__);   \
    case 33: return FN<16, true>(__VA_ARGS__);    \
    default: return cudaErrorInvalidValue;        \
  }

cudaError_t launch_agg_lines(const KParams &k, const Buffers &b, int nf, bool spill8, cudaStream_t s) {
  SGMF_DISPATCH(launch_lines_t, k, b, nf, s)
}

cudaError_t launch_agg_sweep(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  switch (k.DPL) {
    case 2: return launch_sweep_t<4>(k, b, nf, s);
    case 4: return launch_sweep_t<8>(k, b, nf, s);
    case 6: return launch_sweep_t<12>(k, b, nf, s);
    case 8: return launch_sweep_t<16>(k, b, nf, s);
    default: return cudaErrorInvalidValue;
  }
}

int agg_sweep_plan(const KParams &k, int nb, int *slots) {
  switch (k.DPL) {
    case 2: return sweep_plan_t<4>(k, nb, slots);
    case 4: return sweep_plan_t<8>(k, nb, slots);
    case 6: return sweep_plan_t<12>(k, nb, slots);
    case 8: return sweep_plan_t<16>(k, nb, slots);
    default: return 0;
  }
}

cudaError_t launch_agg_rows(const KParams &k, const Buffers &b, int nf, bool spill8, cudaStream_t s) {
  SGMF_DISPATCH(launch_rows_t, k, b, nf, s)
}

}  // namespace sgmf
