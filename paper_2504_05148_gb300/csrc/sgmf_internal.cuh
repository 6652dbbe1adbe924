// sgmf_internal.cuh -- shared declarations of the CUDA library (sm_103a).
//
// Device data layout (all row-major, frame outermost, then y):
//   images          uint8  [F][H][pitch]   pitched copies (pitch % 16 == 0) for TMA
//   d-bar, d-hat    int16  [F][H][W]       -1 = invalid
//   census          u32 (CS 9x7) or u64 (9x7) [F][H][W]
//   box-OR masks    u32    [F][MW][H][W]   bit d of word-plane d/32 set when a
//                                           sparse disparity of the window is d
//   cost C-bar      uint8  [F][H][W][Dp]   Dp = 32 * DPL >= D, cells d >= D hold 0
//   partial sums    u16    [F][H][W][Dp]   one per line family (vertical, two diagonals)
//   spills          uint8/u16 [F][4][line][pos][Dp]  first-direction path costs of a line
// F is the number of frames a context holds (its batch capacity); every
// kernel takes the frame from its last grid dimension.
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <type_traits>
#include <cuda_runtime.h>

#include "sgmf.h"

namespace sgmf {

constexpr int kMaxDisp = 256;
constexpr int kMaxDim = 8192;
// banded mode: the band start is constant on kBandTile x kBandTile pixel tiles
constexpr int kBandTileLog = 3, kBandTile = 1 << kBandTileLog;
constexpr uint32_t kInf = 0x4000u;          // u16 lane value above every real path cost
constexpr uint32_t kInf2 = kInf | (kInf << 16);

enum ErrorCode : int { kErrNone = 0, kErrTimeout = 6 };

// Parameters in the form the kernels use (validated on the host).
struct KParams {
  int W, H, D, Dp, DPL, MW;   // MW = Dp / 32 mask words per pixel
  int pitch;                  // image pitch in bytes
  int p1, p2, q1, q2, a, b;   // alpha = a / b
  int ts, rs, tc, rc, lr;
  int census, semidense, consistency, num_paths, subpixel;
  int nbits;
  int line_warps, cost_px;    // tuning: warps per line-kernel CTA, pixels per cost-kernel CTA
  int sweep;                  // tuning: 1 = row-synchronous sweep instead of the line kernels
  int sweep_cs;               // CTAs per sweep cluster (0: the sweep cannot run this context)
  int parts;                  // tuning: 1 = sweep batches in parts (row kernels on a second stream)
  int band;                   // banded mode: band width B (= Dp); 0 = the plain method
  int tw, th;                 // banded mode: band tiles per row / column
  uint32_t wait_census;       // poll limit of the census kernel's TMA wait (kWaitLimit by default)
  int gate_run;               // with Buffers::gate: a frame runs when its gate word equals this
};

struct Buffers {   // base pointers of frame 0
  uint8_t *imgL, *imgR;       // pitched copies
  int16_t *dbar, *dhat, *dstar, *dprime;
  int16_t *dsub;              // sub-pixel disparity (1/16 px)
  void *censL, *censR;        // u32 or u64 per pixel
  uint32_t *boxS;             // [MW][H][W] box-ORed presence masks, radius r_s
  uint32_t *boxC;             // [MW][H][W] their row ORs only (|x' - x| <= r_c), radius r_c
  uint32_t *boxTmp;           // [F][MW][H][W] r_s row-pass results (scratch of the column pass)
  uint8_t *cost;              // [H][W][Dp]
  uint16_t *part[3];          // [H][W][Dp]
  void *spill;                // 4 regions (vertical, diag, anti-diag, rows) of H*W*Dp elements
  uint16_t *dbg_sum;          // [H][W][Dp] or null
  int *err;                   // device error word
  int16_t *band_lo;           // banded mode: band start per tile, [frame][th][tw] (clamped copy)
  const int *gate;            // per-frame gate words (caller's device memory) or null: every frame runs
};

// per-frame element counts
__host__ __device__ __forceinline__ size_t frame_px(const KParams &k) { return (size_t)k.W * k.H; }
__host__ __device__ __forceinline__ size_t frame_cells(const KParams &k) { return (size_t)k.W * k.H * k.Dp; }

// the buffers of frame f (spill regions hold 2-byte elements at most; the
// kernels that use them offset by the element size they store)
__host__ __device__ __forceinline__ Buffers frame_view(const KParams &k, const Buffers &b, int f) {
  const size_t px = frame_px(k), cells = frame_cells(k);
  Buffers v = b;
  v.imgL = b.imgL + (size_t)f * k.pitch * k.H;
  v.imgR = b.imgR + (size_t)f * k.pitch * k.H;
  v.dbar = b.dbar + f * px;
  v.dhat = b.dhat + f * px;
  v.dstar = b.dstar + f * px;
  v.dprime = b.dprime + f * px;
  v.dsub = b.dsub + f * px;
  const size_t cw = k.census == 1 ? 8 : 4;
  v.censL = static_cast<uint8_t *>(b.censL) + f * px * cw;
  v.censR = static_cast<uint8_t *>(b.censR) + f * px * cw;
  v.boxS = b.boxS + f * px * k.MW;
  v.boxC = b.boxC + f * px * k.MW;
  v.cost = b.cost + f * cells;
  for (int i = 0; i < 3; ++i) v.part[i] = b.part[i] + f * cells;
  v.spill = static_cast<uint8_t *>(b.spill) + f * 4 * cells * 2;
  v.dbg_sum = (b.dbg_sum != nullptr && f == 0) ? b.dbg_sum : nullptr;
  v.band_lo = b.band_lo ? b.band_lo + (size_t)f * k.th * k.tw : nullptr;
  v.gate = b.gate ? b.gate + f : nullptr;
  return v;
}

// Whether the kernels skip a frame: its gate word (gate_f, the frame's own,
// or null) differs from the context's run value.  Every CTA works on one
// frame, so the test is uniform per CTA and comes before any barrier or copy.
__host__ __device__ __forceinline__ bool gated_off(const int *gate_f, int run) {
  return gate_f != nullptr && *gate_f != run;
}

// ---- small device helpers ------------------------------------------------

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
  return __byte_perm(a, b, s);
}

// ---- cost kernels: vector reads of the right census, packed cost bytes ------
template <typename CT>
__device__ __forceinline__ int hamming(CT a, CT b) {
  if constexpr (sizeof(CT) == 4)
    return __popc(a ^ b);
  else
    return __popcll(a ^ b);
}

template <typename CT, int DPL>
struct CostVec {
  // entries per vector load: 16 bytes, or 8 when DPL is not a multiple of 4 words
  static constexpr int VL = sizeof(CT) == 8 ? 2 : (DPL % 4 == 0 ? 4 : 2);
  using V = typename std::conditional<VL * sizeof(CT) == 16, uint4, uint2>::type;
};

template <int DPL>
__device__ __forceinline__ void store_cost_bytes(uint8_t *o, const uint32_t (&b)[DPL]) {
  uint32_t w[(DPL + 3) / 4];
#pragma unroll
  for (int j = 0; j < DPL / 4; ++j)
    w[j] = prmt(prmt(b[4 * j], b[4 * j + 1], 0x1140), prmt(b[4 * j + 2], b[4 * j + 3], 0x1140), 0x5410);
  if constexpr (DPL == 2) {
    *reinterpret_cast<uint16_t *>(o) = (uint16_t)prmt(b[0], b[1], 0x1140);
  } else if constexpr (DPL == 4) {
    *reinterpret_cast<uint32_t *>(o) = w[0];
  } else if constexpr (DPL == 6) {   // 2-byte aligned
    uint16_t *q = reinterpret_cast<uint16_t *>(o);
    q[0] = (uint16_t)prmt(b[0], b[1], 0x1140);
    q[1] = (uint16_t)prmt(b[2], b[3], 0x1140);
    q[2] = (uint16_t)prmt(b[4], b[5], 0x1140);
  } else {
    *reinterpret_cast<uint2 *>(o) = make_uint2(w[0], w[1]);
  }
}


// sticky error word: first error wins
__device__ __forceinline__ void set_error(int *err, int code) {
  atomicCAS(err, 0, code);
}

// ---- mbarrier / TMA (inline PTX) -------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: true when the phase completed, false after `limit` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

constexpr uint32_t kWaitLimit = 1u << 22;   // polls (each try_wait may suspend briefly)

// 1-D bulk copy global -> shared; both addresses 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// order this thread's earlier generic-proxy global writes before later
// async-proxy (bulk copy) reads of the same data
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// order this thread's earlier shared-memory writes before later async-proxy
// (bulk copy) reads of them
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy shared -> global, in the thread's current bulk group; both
// addresses 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(reinterpret_cast<uint64_t>(dst)),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the thread's bulk groups but the newest one have read their shared memory
__device__ __forceinline__ void bulk_wait_read_all_but_one() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
// every bulk group of the thread is complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---- per-device one-time set-up (host) --------------------------------------
// Kernel attributes and device properties are set or read once per device
// ordinal.  The library's entry points may be called from any host thread,
// so the flags are read and written under one process-wide mutex.
std::mutex &setup_mutex();

// runs setup(dev) once for the current device; cudaSuccess afterwards
template <typename F>
inline cudaError_t once_per_device(bool (&done)[64], F &&setup) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(setup_mutex());
  if (done[dev]) return cudaSuccess;
  e = setup(dev);
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

// number of SMs of the current device (looked up once per device)
cudaError_t sm_count(int *out);

// ---- kernel launchers (implemented in the .cu files) -----------------------
struct TmaMaps;   // opaque holder of the two image tensor maps (sgmf_front.cu)

// Every launcher covers frames [0, nf) of the context's buffers.
// C-bar of Eq. 4 by q class (0: d = prior, 1: |d - prior| = 1, 2: farther)
// and Hamming distance H; class 3 (no prior) is the identity, C-bar = H:
//   C-bar = floor(((b - a) H + a q + floor(b / 2)) / b),  q = 0 / q1 / q2.
struct CostTable {
  uint8_t v[4][64];
};
inline CostTable cost_table(const KParams &k) {
  CostTable tab;
  const int qs[3] = {0, k.q1, k.q2};
  for (int c = 0; c < 3; ++c)
    for (int h = 0; h < 64; ++h) {
      const long v = ((long)(k.b - k.a) * h + (long)k.a * qs[c] + k.b / 2) / k.b;
      tab.v[c][h] = (uint8_t)(v > 255 ? 255 : v);
    }
  for (int h = 0; h < 64; ++h) tab.v[3][h] = (uint8_t)h;
  return tab;
}

cudaError_t launch_ingest(const KParams &k, const Buffers &b, int nf, const uint8_t *left,
                          const uint8_t *right, const float *lidar, cudaStream_t s);
// b: the buffers of frame zoff (frame_view), which is the tensor maps' frame zoff
cudaError_t launch_census(const KParams &k, const Buffers &b, int nf, int zoff, const void *tmaL, const void *tmaR,
                          cudaStream_t s);
// box-ORs of the presence masks of the sparse map disp [nf][H][W] (values in
// [0, D) present): radius k.rs into boxS and k.rc into boxC, either may be
// null; tmp holds nf * MW * H * W words per wanted radius
cudaError_t launch_boxor(const KParams &k, int nf, const int16_t *disp, uint32_t *tmp, uint32_t *boxS,
                         uint32_t *boxC, cudaStream_t s, const int *gate = nullptr);
cudaError_t launch_boxor_cols(const KParams &k, int nf, const uint32_t *src, uint32_t *dst, int r, cudaStream_t s,
                              const int *gate = nullptr);
cudaError_t launch_semidense(const KParams &k, const Buffers &b, int nf, cudaStream_t s);
cudaError_t launch_cost(const KParams &k, const Buffers &b, int nf, cudaStream_t s);
cudaError_t launch_agg_lines(const KParams &k, const Buffers &b, int nf, bool spill8, cudaStream_t s);
cudaError_t launch_agg_rows(const KParams &k, const Buffers &b, int nf, bool spill8, cudaStream_t s);
// the six vertical/diagonal directions as two cluster sweeps (k.sweep, clusters of
// k.sweep_cs CTAs); plan: the cluster size for the context's shape and batch capacity nb on
// this device, 0 if none, and in *slots the number of such clusters the device holds at once
cudaError_t launch_agg_sweep(const KParams &k, const Buffers &b, int nf, cudaStream_t s);
int agg_sweep_plan(const KParams &k, int nb, int *slots);
cudaError_t launch_band_clamp(const KParams &k, const Buffers &b, int nf, const int16_t *lo_in, cudaStream_t s);
cudaError_t launch_cost_banded(const KParams &k, const Buffers &b, int nf, cudaStream_t s);
cudaError_t launch_consistency(const KParams &k, const Buffers &b, int nf, int16_t *out, cudaStream_t s);

// host: parameter rules of sgmf_set_params (SGMF_OK or SGMF_ERR_PARAM with a reason)
sgmf_status validate_params(const sgmf_params &p, std::string &why);
// host: message returned by sgmf_last_error(NULL) on this thread
void set_noctx_error(const std::string &msg);

// host: encode the 3-D uint8 tensor map {W, H, frames} of the pitched images
// (driver entry point)
int make_image_tmap(void *tmap_out /* CUtensorMap* */, const uint8_t *base, int W, int H, int pitch,
                    int frames, int box_w, int box_h);

// census tile geometry (shared by host map creation and the kernel)
constexpr int kCenTileW = 64;     // output pixels per tile, x
constexpr int kCenTileH = 16;     // output pixels per tile, y
constexpr int kCenBoxW = 96;      // loaded box: x0-16 .. x0+79 (16-byte aligned start)
constexpr int kCenBoxH = 22;      // loaded box: y0-3 .. y0+18

}  // namespace sgmf
