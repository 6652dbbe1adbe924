// sgmf_aggregate.cu -- SGM path aggregation (Eq. 2), path sum and WTA (Eq. 3).
//
// Lines.  Each of the eight directions of Sec. III runs along a family of
// lines; a line is walked once in each of its two directions by one warp:
//   family 0 (vertical)      line k = column k            down: r=(0,1)   up: r=(0,-1)
//   family 1 (diagonal)      line k: x = (k + y) mod W    down: r=(1,1)   up: r=(-1,-1)
//   family 2 (anti-diagonal) line k: x = (k - y) mod W    down: r=(-1,1)  up: r=(1,-1)
//   rows                     line = row y                 right->left r=(-1,0), left->right r=(1,0)
// With the modulo every diagonal line has exactly H pixels, and a path
// (re)starts where the line wraps, i.e. where p - r leaves the image.
//
// Lanes.  Lane l holds disparities [l*DPL, (l+1)*DPL) as DPL/2 u16x2 words.
// One step of Eq. 2 on a word:
//   t     = viaddmin(vimin3(L(d-1), L(d+1), m + P2 - P1), P1, L(d))
//         = min{ L(d), L(d-1)+P1, L(d+1)+P1, m+P2 }
//   L'(d) = t + C(d) - m                      (one 32-bit add: t >= m per half)
// L(d-1), L(d+1) of the two halves come from byte permutes of neighbouring
// words (and one shuffle each way across lanes); m = min_k L(k) is a
// per-lane u16x2 min followed by one __reduce_min_sync.  Disparities beyond
// D are padding: their cost is raised by kInf so they never reach the min.
//
// Data movement.  Every warp streams its inputs through a private ring of
// shared-memory stages filled by 1-D bulk copies (cp.async.bulk, completion
// on one mbarrier per stage) several steps ahead of the recursion, so the
// sequential walk never waits on global-memory latency.
//
// Sums.  The line kernel writes, per family, the pair sum L_down + L_up
// (u16) of each pixel.  The row kernel adds the two row directions and the
// family sums into S = sum_r L_r, takes d* (Eq. 3) with one warp min per
// pixel, and d' (the disparity of the right view) with a systolic running
// min: the best key of right pixel x' = x - d moves one disparity slot per
// step, so after D steps it has seen S(x'+d, d) for every d.
#include <cstdint>

#include "sgmf_internal.cuh"

namespace sgmf {

constexpr unsigned kFull = 0xffffffffu;

// ---- lane-vector access (shared or global memory, generic pointers) ------------
// u8 cells -> u16x2 words; the pad bytes z (0x40 for d >= D) become the high bytes.
template <int DPL>
__device__ __forceinline__ void unpack_u8(const uint8_t *row, int lane, const uint32_t (&z)[(DPL + 3) / 4],
                                          uint32_t (&w)[DPL / 2]) {
  const uint8_t *p = row + lane * DPL;
  if constexpr (DPL == 2) {
    const uint32_t v = *reinterpret_cast<const uint16_t *>(p);
    w[0] = prmt(v, z[0], 0x5140);
  } else if constexpr (DPL == 4) {
    const uint32_t v = *reinterpret_cast<const uint32_t *>(p);
    w[0] = prmt(v, z[0], 0x5140);
    w[1] = prmt(v, z[0], 0x7362);
  } else if constexpr (DPL == 6) {
    const uint16_t *q = reinterpret_cast<const uint16_t *>(p);
    const uint32_t v0 = q[0], v1 = q[1], v2 = q[2];
    // z[0] holds the pads of cells 0..3, z[1] of cells 4..5 (bytes 0, 1)
    w[0] = prmt(v0, z[0], 0x5140);
    w[1] = prmt(v1, z[0], 0x7160);
    w[2] = prmt(v2, z[1], 0x5140);
  } else {
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    w[0] = prmt(v.x, z[0], 0x5140);
    w[1] = prmt(v.x, z[0], 0x7362);
    w[2] = prmt(v.y, z[1], 0x5140);
    w[3] = prmt(v.y, z[1], 0x7362);
  }
}

// u16x2 words -> u8 cells (every real value is <= 255 when this is used)
template <int DPL>
__device__ __forceinline__ void store_u8(uint8_t *row, int lane, const uint32_t (&w)[DPL / 2]) {
  uint8_t *p = row + lane * DPL;
  if constexpr (DPL == 2) {
    *reinterpret_cast<uint16_t *>(p) = (uint16_t)prmt(w[0], 0, 0x0020);
  } else if constexpr (DPL == 4) {
    *reinterpret_cast<uint32_t *>(p) = prmt(w[0], w[1], 0x6420);
  } else if constexpr (DPL == 6) {
    uint16_t *q = reinterpret_cast<uint16_t *>(p);
    q[0] = (uint16_t)prmt(w[0], 0, 0x0020);
    q[1] = (uint16_t)prmt(w[1], 0, 0x0020);
    q[2] = (uint16_t)prmt(w[2], 0, 0x0020);
  } else {
    *reinterpret_cast<uint2 *>(p) = make_uint2(prmt(w[0], w[1], 0x6420), prmt(w[2], w[3], 0x6420));
  }
}

template <int DPL>
__device__ __forceinline__ void load_u16(const uint16_t *row, int lane, uint32_t (&w)[DPL / 2]) {
  const uint16_t *p = row + lane * DPL;
  if constexpr (DPL == 2) {
    w[0] = *reinterpret_cast<const uint32_t *>(p);
  } else if constexpr (DPL == 4) {
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    w[0] = v.x;
    w[1] = v.y;
  } else if constexpr (DPL == 6) {
    const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
    w[0] = q[0];
    w[1] = q[1];
    w[2] = q[2];
  } else {
    const uint4 v = *reinterpret_cast<const uint4 *>(p);
    w[0] = v.x;
    w[1] = v.y;
    w[2] = v.z;
    w[3] = v.w;
  }
}

template <int DPL>
__device__ __forceinline__ void store_u16(uint16_t *row, int lane, const uint32_t (&w)[DPL / 2]) {
  uint16_t *p = row + lane * DPL;
  if constexpr (DPL == 2) {
    *reinterpret_cast<uint32_t *>(p) = w[0];
  } else if constexpr (DPL == 4) {
    *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
  } else if constexpr (DPL == 6) {
    uint32_t *q = reinterpret_cast<uint32_t *>(p);
    q[0] = w[0];
    q[1] = w[1];
    q[2] = w[2];
  } else {
    *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// spill of a first-direction path cost vector: u8 when every real cost fits
template <int DPL, bool S8>
__device__ __forceinline__ void spill_put(void *base, size_t cell, int lane, const uint32_t (&w)[DPL / 2]) {
  if constexpr (S8)
    store_u8<DPL>(static_cast<uint8_t *>(base) + cell, lane, w);
  else
    store_u16<DPL>(static_cast<uint16_t *>(base) + cell, lane, w);
}

template <int DPL, bool S8>
__device__ __forceinline__ void spill_get(const uint8_t *stage_row, int lane, uint32_t (&w)[DPL / 2]) {
  if constexpr (S8) {
    const uint32_t z[(DPL + 3) / 4] = {};
    unpack_u8<DPL>(stage_row, lane, z, w);
  } else {
    load_u16<DPL>(reinterpret_cast<const uint16_t *>(stage_row), lane, w);
  }
}

// ---- the recursion -----------------------------------------------------------
struct StepConsts {
  uint32_t p1x2;   // P1 in both halves
  uint32_t dpx2;   // (P2 - P1) in both halves
};

// One step of Eq. 2 for the lane's words.  mm = min_k L(p - r, k) in both
// halves; edge_lo / edge_hi are all-ones on lane 0 / lane 31 so that the
// missing neighbours L(-1) and L(Dp) read as 0xffff (they only enter a min).
template <int NW>
__device__ __forceinline__ void sgm_step(uint32_t (&L)[NW], const uint32_t (&C)[NW], uint32_t mm,
                                         const StepConsts &sc, uint32_t edge_lo, uint32_t edge_hi) {
  const uint32_t cap = mm + sc.dpx2;           // m + P2 - P1 per half
  const uint32_t negmm = 0u - mm;
  const uint32_t prev = __shfl_up_sync(kFull, L[NW - 1], 1) | edge_lo;
  const uint32_t next = __shfl_down_sync(kFull, L[0], 1) | edge_hi;
  uint32_t sh[NW + 1];
  sh[0] = prmt(prev, L[0], 0x5432);
#pragma unroll
  for (int i = 1; i < NW; ++i) sh[i] = prmt(L[i - 1], L[i], 0x5432);
  sh[NW] = prmt(L[NW - 1], next, 0x5432);
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const uint32_t t = __viaddmin_u16x2(__vimin3_u16x2(sh[i], sh[i + 1], cap), sc.p1x2, L[i]);
    L[i] = t + C[i] + negmm;
  }
}

// min over all disparities of the warp's vector, returned in both halves
template <int NW>
__device__ __forceinline__ uint32_t warp_min(const uint32_t (&L)[NW]) {
  uint32_t v = L[0];
#pragma unroll
  for (int i = 1; i + 1 < NW; i += 2) v = __vimin3_u16x2(v, L[i], L[i + 1]);
  if constexpr (NW % 2 == 0) v = __vminu2(v, L[NW - 1]);
  v = __vminu2(v, prmt(v, v, 0x1032));
  return __reduce_min_sync(kFull, v);
}

// pad bytes (0x40 = high byte of kInf) of the lane's cells d >= D
template <int DPL>
__device__ __forceinline__ void pad_bytes(int D, int lane, uint32_t (&z)[(DPL + 3) / 4]) {
#pragma unroll
  for (int i = 0; i < (DPL + 3) / 4; ++i) {
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int d = lane * DPL + 4 * i + j;
      if (4 * i + j < DPL && d >= D) v |= 0x40u << (8 * j);
    }
    z[i] = v;
  }
}

// Bounded wait for ring fill g (stage g % S, phase g / S).  The decision is
// warp-uniform.  On a timeout the warp flags the error, gives every fill it
// has issued (g .. issued-1) a second bounded wait, and reports false so that
// the caller returns.
template <int S>
__device__ __forceinline__ bool ring_wait(uint64_t *bars, int g, int issued, int *err) {
  const bool ok = mbar_wait_bounded(&bars[g % S], (uint32_t)(g / S) & 1u, kWaitLimit);
  if (__all_sync(kFull, ok)) return true;
  if ((threadIdx.x & 31) == 0) set_error(err, kErrTimeout);
  for (int h = g; h < issued; ++h) mbar_wait_bounded(&bars[h % S], (uint32_t)(h / S) & 1u, kWaitLimit);
  return false;
}

// ---- vertical and diagonal families -------------------------------------------
struct LineArgs {
  KParams k;
  const uint8_t *cost;
  uint16_t *part[3];
  void *spill;            // [3][W][H][Dp] elements
  int *err;
  StepConsts sc;
};

template <int DPL, bool S8>
struct LineCfg {
  static constexpr int Dp = 32 * DPL;
  static constexpr int K = DPL == 2 ? 16 : (DPL == 4 ? 8 : 4);   // rows per stage
  static constexpr int S = 4;                                      // stages per warp
  static constexpr int SB = S8 ? 1 : 2;                            // spill bytes per cell
  static constexpr int kCost = K * Dp;
  static constexpr int kStage = kCost + K * Dp * SB;
  static constexpr int kWarp = S * kStage;
  static constexpr int kWarps = 4;
  static constexpr int kSmem = kWarps * kWarp + kWarps * S * 8;
};

// x of line k at row y in family fam
__device__ __forceinline__ int line_x(int fam, int k, int y, int W) {
  if (fam == 0) return k;
  int x = (fam == 1 ? k + y : k - y) % W;
  return x < 0 ? x + W : x;
}

template <int DPL, bool S8>
__global__ void __launch_bounds__(128) k_agg_lines(const __grid_constant__ LineArgs a) {
  using CF = LineCfg<DPL, S8>;
  constexpr int NW = DPL / 2, K = CF::K, S = CF::S, Dp = CF::Dp;
  extern __shared__ __align__(128) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int line = blockIdx.x * CF::kWarps + warp;
  const int fam = blockIdx.y;
  const int W = a.k.W, H = a.k.H;
  if (line >= W) return;                  // warps are independent: no block barrier below
  uint8_t *ring = smem + warp * CF::kWarp;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + CF::kWarps * CF::kWarp) + warp * S;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  uint32_t z[(DPL + 3) / 4];
  pad_bytes<DPL>(a.k.D, lane, z);
  const uint32_t edge_lo = lane == 0 ? 0xffffffffu : 0u, edge_hi = lane == 31 ? 0xffffffffu : 0u;
  const StepConsts sc = a.sc;
  const size_t spill_line = ((size_t)fam * W + line) * (size_t)H * Dp;   // elements
  const int nch = (H + K - 1) / K;
  // fill of ring slot g: chunk g (down) or g - nch (up); rows of the cost volume,
  // plus, going up, the spilled L_down rows of the chunk (one contiguous copy)
  auto issue = [&](int g) {
    const bool up = g >= nch;
    const int c = up ? g - nch : g;
    const int stage = g % S;
    uint8_t *st = ring + stage * CF::kStage;
    int y_lo, n;
    if (!up) {
      y_lo = c * K;
      n = min(K, H - y_lo);
    } else {
      const int y_hi = H - 1 - c * K;
      y_lo = max(0, y_hi - K + 1);
      n = y_hi - y_lo + 1;
    }
    if (lane == 0) mbar_expect_tx(&bars[stage], (uint32_t)(n * Dp * (up ? 1 + CF::SB : 1)));
    __syncwarp();
    if (lane < n) {
      const int y = y_lo + lane;
      bulk_g2s(st + lane * Dp, a.cost + ((size_t)y * W + line_x(fam, line, y, W)) * Dp, Dp, &bars[stage]);
    }
    if (up && lane == 31)
      bulk_g2s(st + CF::kCost, static_cast<const uint8_t *>(a.spill) + (spill_line + (size_t)y_lo * Dp) * CF::SB,
               (uint32_t)(n * Dp * CF::SB), &bars[stage]);
  };

  uint32_t L[NW], C[NW];
  uint32_t mm = 0;
  // path segments: a line restarts where it wraps around the image border
  const int x_top = line_x(fam, line, 0, W), x_bot = line_x(fam, line, H - 1, W);
  const int seg_full = fam == 0 ? H : W;
  // ---- down: r = (0,1), (1,1), (-1,1) ----
  {
    int pos = 0, seg = fam == 0 ? H : (fam == 1 ? W - x_top : x_top + 1);
    uint8_t *sp = static_cast<uint8_t *>(a.spill) + spill_line * CF::SB;
    for (int g = 0; g < S - 1 && g < nch; ++g) issue(g);
    for (int c = 0; c < nch; ++c) {
      if (c + S - 1 < nch) issue(c + S - 1);
      if (!ring_wait<S>(bars, c, min(c + S, nch), a.err)) return;
      const uint8_t *st = ring + (c % S) * CF::kStage;
      const int n = min(K, H - c * K);
      for (int r = 0; r < n; ++r) {
        unpack_u8<DPL>(st + r * Dp, lane, z, C);
        if (pos == 0) {
#pragma unroll
          for (int i = 0; i < NW; ++i) L[i] = C[i];
        } else {
          sgm_step<NW>(L, C, mm, sc, edge_lo, edge_hi);
        }
        if (++pos == seg) {
          pos = 0;
          seg = seg_full;
        }
        mm = warp_min<NW>(L);
        if constexpr (S8)
          store_u8<DPL>(sp, lane, L);
        else
          store_u16<DPL>(reinterpret_cast<uint16_t *>(sp), lane, L);
        sp += Dp * CF::SB;
      }
      __syncwarp();
    }
  }
  // the spilled L_down rows are read back by bulk copies (async proxy)
  fence_proxy_async_global();
  __syncwarp();
  // ---- up: r = (0,-1), (-1,-1), (1,-1); emit L_down + L_up ----
  {
    uint16_t *part = a.part[fam];
    int pos = 0, seg = fam == 0 ? H : (fam == 1 ? x_bot + 1 : W - x_bot);
    int x = x_bot;
    for (int g = nch; g < nch + S - 1 && g < 2 * nch; ++g) issue(g);
    for (int c = 0; c < nch; ++c) {
      const int g = nch + c;
      if (g + S - 1 < 2 * nch) issue(g + S - 1);
      if (!ring_wait<S>(bars, g, nch + min(c + S, nch), a.err)) return;
      const uint8_t *st = ring + (g % S) * CF::kStage;
      const int y_hi = H - 1 - c * K, y_lo = max(0, y_hi - K + 1);
      for (int y = y_hi; y >= y_lo; --y) {
        const int r = y - y_lo;
        unpack_u8<DPL>(st + r * Dp, lane, z, C);
        if (pos == 0) {
#pragma unroll
          for (int i = 0; i < NW; ++i) L[i] = C[i];
        } else {
          sgm_step<NW>(L, C, mm, sc, edge_lo, edge_hi);
        }
        if (++pos == seg) {
          pos = 0;
          seg = seg_full;
        }
        mm = warp_min<NW>(L);
        uint32_t Ld[NW];
        spill_get<DPL, S8>(st + CF::kCost + r * Dp * CF::SB, lane, Ld);
#pragma unroll
        for (int i = 0; i < NW; ++i) Ld[i] += L[i];
        store_u16<DPL>(part + (size_t)(y * W + x) * Dp, lane, Ld);
        if (fam == 1) x = x == 0 ? W - 1 : x - 1;
        else if (fam == 2) x = x == W - 1 ? 0 : x + 1;
      }
      __syncwarp();
    }
  }
}

// ---- rows, path sum and WTA ----------------------------------------------------
// One CTA per image row, two warps meeting in the middle.  Warp 0 walks
// left -> right (r = (1,0)), warp 1 right -> left (r = (-1,0)), both from the
// start.  Each warp spills its path costs for the half it reaches first
// (warp 0: x < xm, warp 1: x >= xm) and, on the half it reaches second,
// reads the other warp's spilled costs (after that warp has published its
// progress), adds the line-family sums into S, and takes d* and d' there.
// The right-view keys of pixels x' whose diagonal crosses xm are merged in
// shared memory at the end.
struct RowArgs {
  KParams k;
  const uint8_t *cost;
  const uint16_t *part[3];
  int nparts;
  void *spill;            // [H][W][Dp] elements
  int16_t *dstar, *dprime;
  uint16_t *dbg_sum;
  int *err;
  StepConsts sc;
};

template <int DPL, bool S8>
struct RowCfg {
  static constexpr int Dp = 32 * DPL;
  static constexpr int K = DPL == 2 ? 8 : 4;    // pixels per stage
  static constexpr int S = 4;
  static constexpr int SB = S8 ? 1 : 2;
  static constexpr int kCost = K * Dp;
  static constexpr int kSpill = K * Dp * SB;
  static constexpr int kPart = K * Dp * 2;
  static constexpr int kStage = kCost + kSpill + 3 * kPart;
  static constexpr int kWarp = S * kStage;
  static constexpr int kSmem = 2 * kWarp + 2 * S * 8 + kMaxDisp * 4 + 16;
};

__device__ __forceinline__ bool wait_progress(volatile int *flag, int need, int *err) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    if (*flag >= need) return true;
    __nanosleep(64);
  }
  set_error(err, kErrTimeout);
  return false;
}

template <int DPL, bool S8>
__device__ __forceinline__ bool row_half_walk(const RowArgs &a, int dir, uint8_t *ring, uint64_t *bars,
                                              volatile int *prog, uint32_t *merge, int y, int xm) {
  using CF = RowCfg<DPL, S8>;
  constexpr int NW = DPL / 2, K = CF::K, S = CF::S, Dp = CF::Dp;
  const int lane = threadIdx.x & 31;
  const int W = a.k.W, D = a.k.D;
  const bool fwd = dir == 0;
  // first half: the pixels this warp reaches first; second half: the rest
  const int n1 = fwd ? xm : W - xm, n2 = W - n1;
  const int c1 = (n1 + K - 1) / K, c2 = (n2 + K - 1) / K, nch = c1 + c2;
  const size_t row = (size_t)y * W;
  uint8_t *spill = static_cast<uint8_t *>(a.spill);
  uint32_t z[(DPL + 3) / 4];
  pad_bytes<DPL>(D, lane, z);
  const uint32_t edge_lo = lane == 0 ? 0xffffffffu : 0u, edge_hi = lane == 31 ? 0xffffffffu : 0u;
  const StepConsts sc = a.sc;
  // chunk c covers walk steps [s_lo, s_hi); walk step s is pixel x = s (fwd) or W-1-s
  auto chunk = [&](int c, int &x_lo, int &n, bool &second) {
    int s_lo, s_hi;
    if (c < c1) {
      s_lo = c * K;
      s_hi = min(n1, s_lo + K);
      second = false;
    } else {
      s_lo = n1 + (c - c1) * K;
      s_hi = min(W, s_lo + K);
      second = true;
    }
    n = s_hi - s_lo;
    x_lo = fwd ? s_lo : W - s_hi;
  };
  auto issue = [&](int g) -> bool {
    int x_lo, n;
    bool second;
    chunk(g, x_lo, n, second);
    const int stage = g % S;
    uint8_t *st = ring + stage * CF::kStage;
    const size_t cell = (row + x_lo) * Dp;
    if (second && g == c1) {
      // the other warp must have spilled its whole first half: the first
      // chunk of this warp's second half is the last one it stores
      bool ok = true;
      if (lane == 0) {
        ok = wait_progress(&prog[fwd ? 1 : 0], 1, a.err);
        __threadfence_block();          // pairs with the writer's fence before its flag store
        fence_proxy_async_global();     // ... and orders the flag read before the bulk copies
      }
      if (!__shfl_sync(kFull, (int)ok, 0)) return false;
    }
    const uint32_t bytes = (uint32_t)(n * Dp * (second ? 1 + CF::SB + 2 * a.nparts : 1));
    if (lane == 0) mbar_expect_tx(&bars[stage], bytes);
    __syncwarp();
    if (lane == 1) bulk_g2s(st, a.cost + cell, (uint32_t)(n * Dp), &bars[stage]);
    if (second) {
      // issued by lane 0, the lane that observed the other warp's progress
      if (lane == 0) bulk_g2s(st + CF::kCost, spill + cell * CF::SB, (uint32_t)(n * Dp * CF::SB), &bars[stage]);
      if (lane >= 2 && lane < 2 + a.nparts)
        bulk_g2s(st + CF::kCost + CF::kSpill + (lane - 2) * CF::kPart, a.part[lane - 2] + cell,
                 (uint32_t)(n * Dp * 2), &bars[stage]);
    }
    return true;
  };
  // key bytes: b0/b1 = disparities of the word's halves, b2/b3 = 0xff on padding
  uint32_t kb[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const int d0 = lane * DPL + 2 * i;
    kb[i] = (uint32_t)(d0 & 0xff) | ((uint32_t)((d0 + 1) & 0xff) << 8) | (d0 >= D ? 0xff0000u : 0u) |
            (d0 + 1 >= D ? 0xff000000u : 0u);
  }
  const int lastLane = (D - 1) / DPL, lastSlot = (D - 1) % DPL;
  const int mbase = xm - D + 1;           // merge slot i holds right pixel mbase + i
  uint32_t L[NW], C[NW];
  uint32_t mm = 0;
  uint32_t acc[DPL];
#pragma unroll
  for (int j = 0; j < DPL; ++j) acc[j] = 0xffffffffu;
  int issued = 0;
  // on a failed progress wait, let the fills already issued (c .. issued-1) land first
  auto drain = [&](int c) {
    for (int h = c; h < issued; ++h) mbar_wait_bounded(&bars[h % S], (uint32_t)(h / S) & 1u, kWaitLimit);
  };
  // Fills run up to S-1 chunks ahead, except that no second-half fill (which
  // waits for the other warp's first half) is issued before this warp has
  // published its own first half: each warp's first half waits on nothing,
  // so neither warp can wait on the other in a cycle.
  auto may_issue = [&](int c) { return issued < nch && issued < c + S && (issued < c1 || c >= c1); };
  for (int c = 0; c < nch; ++c) {
    while (may_issue(c)) {
      if (!issue(issued)) {
        drain(c);
        return false;
      }
      ++issued;
    }
    if (!ring_wait<S>(bars, c, issued, a.err)) return false;
    const uint8_t *st = ring + (c % S) * CF::kStage;
    int x_lo, n;
    bool second;
    chunk(c, x_lo, n, second);
    for (int i = 0; i < n; ++i) {
      const int r = fwd ? i : n - 1 - i;      // stage rows are in increasing x
      const int x = x_lo + r;
      unpack_u8<DPL>(st + r * Dp, lane, z, C);
      if (x == (fwd ? 0 : W - 1)) {
#pragma unroll
        for (int w = 0; w < NW; ++w) L[w] = C[w];
      } else {
        sgm_step<NW>(L, C, mm, sc, edge_lo, edge_hi);
      }
      mm = warp_min<NW>(L);
      if (!second) {
        if constexpr (S8)
          store_u8<DPL>(spill + (row + x) * Dp, lane, L);
        else
          store_u16<DPL>(reinterpret_cast<uint16_t *>(spill) + (row + x) * Dp, lane, L);
        continue;
      }
      uint32_t Sm[NW], T[NW];
      spill_get<DPL, S8>(st + CF::kCost + r * Dp * CF::SB, lane, Sm);
#pragma unroll
      for (int w = 0; w < NW; ++w) Sm[w] += L[w];
      for (int j = 0; j < a.nparts; ++j) {
        load_u16<DPL>(reinterpret_cast<const uint16_t *>(st + CF::kCost + CF::kSpill + j * CF::kPart) + r * Dp,
                      lane, T);
#pragma unroll
        for (int w = 0; w < NW; ++w) Sm[w] += T[w];
      }
      if (a.dbg_sum != nullptr) store_u16<DPL>(a.dbg_sum + (row + x) * Dp, lane, Sm);
      uint32_t key[DPL];
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        key[2 * w] = prmt(Sm[w], kb[w], 0x6104);
        key[2 * w + 1] = prmt(Sm[w], kb[w], 0x7325);
      }
      uint32_t best = key[0];
#pragma unroll
      for (int j = 1; j < DPL; ++j) best = min(best, key[j]);
      best = __reduce_min_sync(kFull, best);
      if (lane == 0) a.dstar[row + x] = (int16_t)(best & 0xffu);
      if (fwd) {
        // slot d holds right pixel x - d; shift up, fold in S(x, d)
        uint32_t in = __shfl_up_sync(kFull, acc[DPL - 1], 1);
        if (lane == 0) in = 0xffffffffu;
#pragma unroll
        for (int j = DPL - 1; j > 0; --j) acc[j] = min(acc[j - 1], key[j]);
        acc[0] = min(in, key[0]);
        const int xr = x - (D - 1);
        if (lane == lastLane && xr >= 0) {
          uint32_t v = acc[0];
#pragma unroll
          for (int j = 1; j < DPL; ++j)
            if (j == lastSlot) v = acc[j];
          if (xr >= xm)
            a.dprime[row + xr] = (int16_t)(v & 0xffu);
          else
            atomicMin(&merge[xr - mbase], v);
        }
      } else {
        // slot d holds right pixel x - d; shift down, fold in S(x, d)
        uint32_t in = __shfl_down_sync(kFull, acc[0], 1);
        if (lane == 31) in = 0xffffffffu;
#pragma unroll
        for (int j = 0; j + 1 < DPL; ++j) acc[j] = min(acc[j + 1], key[j]);
        acc[DPL - 1] = min(in, key[DPL - 1]);
        if (lane == 0) {
          if (x + D - 1 < xm)
            a.dprime[row + x] = (int16_t)(acc[0] & 0xffu);
          else
            atomicMin(&merge[x - mbase], acc[0]);
        }
      }
    }
    __syncwarp();
    if (c + 1 == c1) {
      // publish the spilled first half to the other warp
      fence_proxy_async_global();
      __threadfence_block();
      __syncwarp();
      if (lane == 0) *(fwd ? &prog[0] : &prog[1]) = 1;
    }
  }
  if (fwd) {
    // right pixels x' = W-1-d whose diagonal leaves the image: slot d
#pragma unroll
    for (int j = 0; j < DPL; ++j) {
      const int d = lane * DPL + j, xr = W - 1 - d;
      if (d < D - 1 && xr >= 0) {
        if (xr >= xm)
          a.dprime[row + xr] = (int16_t)(acc[j] & 0xffu);
        else
          atomicMin(&merge[xr - mbase], acc[j]);
      }
    }
  }
  return true;
}

template <int DPL, bool S8>
__global__ void __launch_bounds__(64) k_agg_rows(const __grid_constant__ RowArgs a) {
  using CF = RowCfg<DPL, S8>;
  constexpr int S = CF::S;
  extern __shared__ __align__(128) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.x, W = a.k.W, D = a.k.D;
  uint8_t *ring = smem + warp * CF::kWarp;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * CF::kWarp) + warp * S;
  uint32_t *merge = reinterpret_cast<uint32_t *>(smem + 2 * CF::kWarp + 2 * S * 8);
  volatile int *prog = reinterpret_cast<volatile int *>(merge + kMaxDisp);
  const int xm = W / 2;
  for (int i = threadIdx.x; i < kMaxDisp; i += blockDim.x) merge[i] = 0xffffffffu;
  if (threadIdx.x < 2) prog[threadIdx.x] = 0;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = row_half_walk<DPL, S8>(a, warp, ring, bars, prog, merge, y, xm);
  __syncthreads();
  // right pixels whose diagonal crosses xm: both warps contributed
  const int ok_all = __syncthreads_and(ok ? 1 : 0);
  if (ok_all && warp == 0) {
    for (int i = lane; i < D - 1; i += 32) {
      const int xr = xm - D + 1 + i;
      if (xr >= 0 && xr < xm) a.dprime[(size_t)y * W + xr] = (int16_t)(merge[i] & 0xffu);
    }
  }
}

template <int DPL, bool S8>
static cudaError_t launch_lines_t(const KParams &k, const Buffers &b, cudaStream_t s) {
  using CF = LineCfg<DPL, S8>;
  static bool attr[64] = {};   // per device: opt in to more than 48 KB of dynamic shared memory
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_agg_lines<DPL, S8>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::kSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  LineArgs a;
  a.k = k;
  a.cost = b.cost;
  for (int i = 0; i < 3; ++i) a.part[i] = b.part[i];
  a.spill = b.spill;
  a.err = b.err;
  a.sc.p1x2 = (uint32_t)k.p1 * 0x10001u;
  a.sc.dpx2 = (uint32_t)(k.p2 - k.p1) * 0x10001u;
  dim3 grid((k.W + CF::kWarps - 1) / CF::kWarps, k.num_paths == 8 ? 3 : 1);
  k_agg_lines<DPL, S8><<<grid, 32 * CF::kWarps, CF::kSmem, s>>>(a);
  return cudaGetLastError();
}

template <int DPL, bool S8>
static cudaError_t launch_rows_t(const KParams &k, const Buffers &b, cudaStream_t s) {
  using CF = RowCfg<DPL, S8>;
  static bool attr[64] = {};   // per device: opt in to more than 48 KB of dynamic shared memory
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_agg_rows<DPL, S8>, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::kSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  RowArgs a;
  a.k = k;
  a.cost = b.cost;
  for (int i = 0; i < 3; ++i) a.part[i] = b.part[i];
  a.nparts = k.num_paths == 8 ? 3 : 1;
  const size_t region = (size_t)k.W * k.H * k.Dp * (S8 ? 1 : 2);
  a.spill = static_cast<uint8_t *>(b.spill) + 3 * region;
  a.dstar = b.dstar;
  a.dprime = b.dprime;
  a.dbg_sum = b.dbg_sum;
  a.err = b.err;
  a.sc.p1x2 = (uint32_t)k.p1 * 0x10001u;
  a.sc.dpx2 = (uint32_t)(k.p2 - k.p1) * 0x10001u;
  k_agg_rows<DPL, S8><<<k.H, 64, CF::kSmem, s>>>(a);
  return cudaGetLastError();
}

#define SGMF_DISPATCH(FN, ...)                   \
  switch (k.DPL * 2 + (spill8 ? 1 : 0)) {        \
    case 4: return FN<2, false>(__VA_ARGS__);    \
    case 5: return FN<2, true>(__VA_ARGS__);     \
    case 8: return FN<4, false>(__VA_ARGS__);    \
    case 9: return FN<4, true>(__VA_ARGS__);     \
    case 12: return FN<6, false>(__VA_ARGS__);   \
    case 13: return FN<6, true>(__VA_ARGS__);    \
    case 16: return FN<8, false>(__VA_ARGS__);   \
    case 17: return FN<8, true>(__VA_ARGS__);    \
    default: return cudaErrorInvalidValue;       \
  }

cudaError_t launch_agg_lines(const KParams &k, const Buffers &b, bool spill8, cudaStream_t s) {
  SGMF_DISPATCH(launch_lines_t, k, b, s)
}

cudaError_t launch_agg_rows(const KParams &k, const Buffers &b, bool spill8, cudaStream_t s) {
  SGMF_DISPATCH(launch_rows_t, k, b, s)
}

}  // namespace sgmf
