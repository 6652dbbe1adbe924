// sgmf_probe.cu -- issue rates of the integer instructions the pipeline is
// built from, measured on the device at hand (sgmf_measure_rates).
//
// The roofline of the integer path needs the rate at which an SM issues the
// u16x2 min of the path recursion and the population count of the Hamming
// cost.  Each probe kernel runs one CTA per SM (its dynamic shared memory
// keeps a second CTA off the SM) of 1024 threads, every thread driving eight
// independent chains of one instruction kind; the CTA's clock64 span gives
// lanes per clock per SM, independent of the clock the GPU runs at.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "sgmf.h"
#include "sgmf_internal.cuh"

namespace sgmf {

enum ProbeOp : int { kOpMin3 = 0, kOpAddMin = 1, kOpIadd = 2, kOpPopc = 3, kOpPrmt = 4, kNumOps = 5 };

constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 8;     // independent chains a thread
constexpr int kProbeUnroll = 16;    // steps of every chain per loop iteration
constexpr int kProbeSmem = 120 * 1024;
constexpr int kProbeMaxSms = 1024;

static __device__ unsigned long long g_probe_cycles[kProbeMaxSms];
static __device__ uint32_t g_probe_sink[1];

template <int OP>
__device__ __forceinline__ uint32_t probe_step(uint32_t a, uint32_t b, uint32_t c) {
  if constexpr (OP == kOpMin3) return __vimin3_u16x2(a, b, c);
  if constexpr (OP == kOpAddMin) return __viaddmin_u16x2(a, b, c);
  if constexpr (OP == kOpIadd) return a + b;
  if constexpr (OP == kOpPopc) return (uint32_t)__popc(b);
  return __byte_perm(a, b, 0x5432);
}

// every chain j takes its second (and third) operand from chains j+1, j+2 of
// the previous step, so no operand is loop-invariant and nothing folds
template <int OP>
__global__ void __launch_bounds__(kProbeThreads, 1) k_probe(uint32_t seed, int iters) {
  extern __shared__ uint32_t keep_one_cta_per_sm[];
  uint32_t v[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) v[j] = (seed ^ (threadIdx.x * 0x9e3779b9u)) + 0x01000100u * (j + 1);
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kProbeChains; ++j)
        v[j] = probe_step<OP>(v[j], v[(j + 1) % kProbeChains], v[(j + 2) % kProbeChains]);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t r = 0;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) r ^= v[j];
  if (r == seed) g_probe_sink[0] = r + keep_one_cta_per_sm[0];   // keeps the chains live
  if (threadIdx.x == 0) g_probe_cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

template <int OP>
static cudaError_t run_probe(int sms, int iters, double *lanes_per_clk) {
  static bool done[64] = {};
  cudaError_t e = once_per_device(done, [](int) {
    return cudaFuncSetAttribute(k_probe<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
  });
  if (e != cudaSuccess) return e;
  k_probe<OP><<<sms, kProbeThreads, kProbeSmem>>>(0x12345u + OP, iters);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<unsigned long long> cyc(sms);
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(cyc.data(), g_probe_cycles, sizeof(unsigned long long) * sms);
  if (e != cudaSuccess) return e;
  // the median CTA (one per SM)
  std::sort(cyc.begin(), cyc.end());
  const double c = (double)std::max<unsigned long long>(cyc[sms / 2], 1);
  *lanes_per_clk = (double)kProbeThreads * iters * kProbeUnroll * kProbeChains / c;
  return cudaSuccess;
}

}  // namespace sgmf

using namespace sgmf;

extern "C" sgmf_status sgmf_measure_rates(int iters, sgmf_rates *out) {
  if (!out || iters < 1 || iters > (1 << 20)) {
    set_noctx_error("sgmf_measure_rates: need out != NULL and 1 <= iters <= 2^20");
    return SGMF_ERR_ARG;
  }
  int sms = 0;
  cudaError_t e = sm_count(&sms);
  if (e == cudaSuccess && (sms < 1 || sms > kProbeMaxSms)) e = cudaErrorInvalidDevice;
  double r[kNumOps] = {};
  if (e == cudaSuccess) e = run_probe<kOpMin3>(sms, iters, &r[kOpMin3]);
  if (e == cudaSuccess) e = run_probe<kOpAddMin>(sms, iters, &r[kOpAddMin]);
  if (e == cudaSuccess) e = run_probe<kOpIadd>(sms, iters, &r[kOpIadd]);
  if (e == cudaSuccess) e = run_probe<kOpPopc>(sms, iters, &r[kOpPopc]);
  if (e == cudaSuccess) e = run_probe<kOpPrmt>(sms, iters, &r[kOpPrmt]);
  if (e != cudaSuccess) {
    set_noctx_error(std::string("sgmf_measure_rates: ") + cudaGetErrorString(e));
    return SGMF_ERR_CUDA;
  }
  out->sms = sms;
  out->min3_u16x2 = r[kOpMin3];
  out->addmin_u16x2 = r[kOpAddMin];
  out->iadd = r[kOpIadd];
  out->popc = r[kOpPopc];
  out->prmt = r[kOpPrmt];
  return SGMF_OK;
}
