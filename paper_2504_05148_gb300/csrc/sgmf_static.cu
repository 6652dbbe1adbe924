// sgmf_static.cu -- a context-free, allocation-free entry point for the
// stereo-LiDAR consistency stage.
//
// Some callers cannot allocate device memory at the point where they want
// this stage: code running under an allocator they do not own (a memory pool
// that is already carved up, a real-time loop that forbids cudaMalloc after
// start-up, a plugin host that hands out only input and output buffers).
// sgmf_check_static serves them: it takes caller-owned inputs and output and
// keeps its working masks in one file-scope device array that every GPU
// loading this library holds until the process exits.  It calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array is shared by every call: calls that overlap on the GPU (other
// streams, other host threads) race on it.  Every word a call reads is
// written earlier in the same call, so nothing carries over between calls.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "sgmf.h"
#include "sgmf_internal.cuh"

namespace sgmf {

// 8 Mi 32-bit words (32 MiB): three [MW][H][W] planes (d-bar in the first,
// the second spare, the r_c row ORs of the presence masks in the third,
// which the check kernel ORs over the window's rows); with D <= 128 (MW <= 4) that holds
// frames of up to about 700 000 pixels.
constexpr size_t kStaticScratchWords = size_t(8) << 20;
static __device__ __align__(256) uint32_t g_check_scratch[kStaticScratchWords];

// d-bar of the raw LiDAR map (the same ingest rule as the pipeline:
// rint(f) for finite f > 0 with rint(f) <= D-1, else -1)
__global__ void __launch_bounds__(256) k_static_dbar(int W, int H, int D, const float *__restrict__ lidar,
                                                     int16_t *__restrict__ dbar) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= W || y >= H) return;
  const size_t p = (size_t)y * W + x;
  int v = -1;
  if (lidar != nullptr) {
    const float f = lidar[p];
    if (isfinite(f) && f > 0.0f) {
      const float r = rintf(f);
      if (r <= (float)(D - 1)) v = (int)r;
    }
  }
  dbar[p] = (int16_t)v;
}

namespace {
std::mutex g_addr_mu;
uint32_t *g_addr[64] = {};            // device address of g_check_scratch per device ordinal
unsigned long long g_ctx_id[64] = {}; // the context that address belongs to

sgmf_status fail_static(sgmf_status s, const std::string &msg) {
  set_noctx_error(msg);
  return s;
}

// Unique id of the calling thread's current CUDA context, 0 when there is
// none or it is no longer valid (driver entry points, so that the library
// needs no link against the driver library).
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrentFn)(CUcontext *);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long *);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {   // under g_addr_mu
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(p);
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current == nullptr || get_id == nullptr || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device, looked up
// with that device current and cached per device.  The cache belongs to the
// context it was read in: when the current context is another one (the
// device was reset with cudaDeviceReset and its primary context made anew),
// the address is looked up again.
cudaError_t scratch_address(uint32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  const unsigned long long id = g_addr[dev] != nullptr ? current_context_id() : 0;
  if (g_addr[dev] == nullptr || id == 0 || id != g_ctx_id[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_check_scratch);   // makes the device's context current if needed
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<uint32_t *>(ptr);
    g_ctx_id[dev] = current_context_id();
  }
  *out = g_addr[dev];
  return cudaSuccess;
}
}  // namespace

}  // namespace sgmf

using namespace sgmf;

extern "C" sgmf_status sgmf_check_static(int width, int height, int max_disp, const sgmf_params *p,
                                         const int16_t *dstar, const int16_t *dprime,
                                         const float *sparse_lidar_disp, int16_t *out_disp, void *cuda_stream) {
  if (!p || !dstar || !dprime || !out_disp)
    return fail_static(SGMF_ERR_ARG, "sgmf_check_static: NULL parameter, disparity or output pointer");
  if (width < 1 || height < 1 || width > kMaxDim || height > kMaxDim || max_disp < 1 || max_disp > kMaxDisp)
    return fail_static(SGMF_ERR_SHAPE, "sgmf_check_static: need 1 <= width, height <= 8192, 1 <= max_disp <= 256");
  std::string why;
  if (validate_params(*p, why) != SGMF_OK) return fail_static(SGMF_ERR_PARAM, "sgmf_check_static: " + why);
  if (p->subpixel != 0)
    return fail_static(SGMF_ERR_PARAM, "sgmf_check_static: subpixel must be 0 (integer output only)");
  KParams k{};
  k.W = width;
  k.H = height;
  k.D = max_disp;
  k.DPL = max_disp <= 64 ? 2 : max_disp <= 128 ? 4 : max_disp <= 192 ? 6 : 8;
  k.Dp = 32 * k.DPL;
  k.MW = k.Dp / 32;
  k.tc = p->tc;
  k.rc = p->rc;
  k.lr = p->lr_max_diff;
  k.consistency = p->consistency;
  const size_t plane = (size_t)width * height * k.MW;
  if (3 * plane > kStaticScratchWords) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "sgmf_check_static: %d x %d with D = %d needs %zu scratch words, the static array holds %zu",
             width, height, max_disp, 3 * plane, kStaticScratchWords);
    return fail_static(SGMF_ERR_SHAPE, buf);
  }
  uint32_t *scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return fail_static(SGMF_ERR_CUDA, std::string("sgmf_check_static: cudaGetSymbolAddress failed: ") +
                                          cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // d-bar (int16, the first half plane), a spare plane, the r_c row ORs
  int16_t *dbar = reinterpret_cast<int16_t *>(scratch);
  uint32_t *tmp = scratch + plane, *box = scratch + 2 * plane;
  dim3 grid((width + 31) / 32, (height + 7) / 8);
  k_static_dbar<<<grid, 256, 0, s>>>(width, height, max_disp, sparse_lidar_disp, dbar);
  e = cudaGetLastError();
  if (e == cudaSuccess && (k.consistency == SGMF_CHECK_STEREO_LIDAR || k.consistency == SGMF_CHECK_LIDAR))
    e = launch_boxor(k, 1, dbar, tmp, nullptr, box, s);
  if (e == cudaSuccess) {
    Buffers b{};
    b.dstar = const_cast<int16_t *>(dstar);
    b.dprime = const_cast<int16_t *>(dprime);
    b.boxC = box;
    e = launch_consistency(k, b, 1, out_disp, s);
  }
  if (e != cudaSuccess)
    return fail_static(SGMF_ERR_CUDA, std::string("sgmf_check_static: launch failed: ") + cudaGetErrorString(e));
  return SGMF_OK;
}
