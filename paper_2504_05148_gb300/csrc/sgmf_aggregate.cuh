// sgmf_aggregate.cuh -- SGM path aggregation (Eq. 2), path sum and WTA (Eq. 3).
//
// Kernel templates; sgmf_agg_cpl*.cu instantiate them per lane width (one
// translation unit each, compiled in parallel) and sgmf_aggregate.cu picks
// the instantiation for a context.
//
// Lines.  Each of the eight directions of Sec. III runs along a family of
// lines; a line is walked once in each of its two directions:
//   family 0 (vertical)      line k = column k            down: r=(0,1)   up: r=(0,-1)
//   family 1 (diagonal)      line k: x = (k + y) mod W    down: r=(1,1)   up: r=(-1,-1)
//   family 2 (anti-diagonal) line k: x = (k - y) mod W    down: r=(-1,1)  up: r=(1,-1)
//   rows                     line = row y                 left->right r=(1,0), right->left r=(-1,0)
// With the modulo every diagonal line has exactly H pixels, and a path
// (re)starts where the line wraps, i.e. where p - r leaves the image.
//
// Lanes.  A group of 16 lanes (half a warp) walks one line; lane j of the
// group holds disparities [j*CPL, (j+1)*CPL) (CPL = Dp/16 cells) as CPL/2
// u16x2 words.  One step of Eq. 2 on a word:
//   t     = viaddmin(vimin3(L(d-1), L(d+1), m + P2 - P1), P1, L(d))
//         = min{ L(d), L(d-1)+P1, L(d+1)+P1, m+P2 }
//   L'(d) = t + C(d) - m                      (one 32-bit add: t >= m per half)
// L(d-1), L(d+1) of the two halves come from byte permutes of neighbouring
// words (and one 16-wide shuffle each way across lanes); m = min_k L(k) is a
// per-lane u16x2 min followed by one __reduce_min_sync over the group.  A path
// start is the same step applied to an all-zero previous vector (with m = 0
// it yields L = C).  Disparities beyond D are padding: their cost is raised
// by kInf so they never reach the min.
//
// Data movement.  Every warp streams its inputs through a private ring of
// shared-memory stages filled by 1-D bulk copies (cp.async.bulk, completion
// on one mbarrier per stage) several steps ahead of the recursion, so the
// sequential walk does not wait on global-memory latency.
//
// Sums.  The line kernel writes, per family, the pair sum L_down + L_up
// (u16) of each pixel.  The row kernel adds the two row directions and the
// family sums into S = sum_r L_r, takes d* (Eq. 3) with one group min per
// pixel, and d' (the disparity of the right view) with a systolic running
// min: the best key of right pixel x' = x - d moves one disparity slot per
// step, so after D steps it has seen S(x'+d, d) for every d.
#pragma once
#include <cstdint>

#include "sgmf_internal.cuh"

namespace sgmf {

constexpr unsigned kFull = 0xffffffffu;

// ---- lane-vector access (shared or global memory, generic pointers) ------------
// CPL u8 cells at p -> CPL/2 u16x2 words; z[j] holds the pad bytes (0x40 for
// d >= D) of cells 4j..4j+3, which become the high bytes.
template <int CPL>
__device__ __forceinline__ void unpack_u8(const uint8_t *p, const uint32_t (&z)[CPL / 4], uint32_t (&w)[CPL / 2]) {
  uint32_t v[CPL / 4];
  if constexpr (CPL == 4) {
    v[0] = *reinterpret_cast<const uint32_t *>(p);
  } else if constexpr (CPL == 8) {
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    v[0] = t.x;
    v[1] = t.y;
  } else if constexpr (CPL == 12) {
    const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
    v[0] = q[0];
    v[1] = q[1];
    v[2] = q[2];
  } else {
    const uint4 t = *reinterpret_cast<const uint4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
#pragma unroll
  for (int j = 0; j < CPL / 4; ++j) {
    w[2 * j] = prmt(v[j], z[j], 0x5140);
    w[2 * j + 1] = prmt(v[j], z[j], 0x7362);
  }
}

// CPL/2 u16x2 words -> CPL u8 cells (every real value is <= 255 when used)
template <int CPL>
__device__ __forceinline__ void store_u8(uint8_t *p, const uint32_t (&w)[CPL / 2]) {
  uint32_t v[CPL / 4];
#pragma unroll
  for (int j = 0; j < CPL / 4; ++j) v[j] = prmt(w[2 * j], w[2 * j + 1], 0x6420);
  if constexpr (CPL == 4) {
    *reinterpret_cast<uint32_t *>(p) = v[0];
  } else if constexpr (CPL == 8) {
    *reinterpret_cast<uint2 *>(p) = make_uint2(v[0], v[1]);
  } else if constexpr (CPL == 12) {
    uint32_t *q = reinterpret_cast<uint32_t *>(p);
    q[0] = v[0];
    q[1] = v[1];
    q[2] = v[2];
  } else {
    *reinterpret_cast<uint4 *>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  }
}

template <int CPL>
__device__ __forceinline__ void load_u16(const uint16_t *p, uint32_t (&w)[CPL / 2]) {
  if constexpr (CPL == 4) {
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    w[0] = t.x;
    w[1] = t.y;
  } else if constexpr (CPL == 12) {
    const uint2 *q = reinterpret_cast<const uint2 *>(p);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const uint2 t = q[j];
      w[2 * j] = t.x;
      w[2 * j + 1] = t.y;
    }
  } else {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int j = 0; j < CPL / 8; ++j) {
      const uint4 t = q[j];
      w[4 * j] = t.x;
      w[4 * j + 1] = t.y;
      w[4 * j + 2] = t.z;
      w[4 * j + 3] = t.w;
    }
  }
}

template <int CPL>
__device__ __forceinline__ void store_u16(uint16_t *p, const uint32_t (&w)[CPL / 2]) {
  if constexpr (CPL == 4) {
    *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
  } else if constexpr (CPL == 12) {
    uint2 *q = reinterpret_cast<uint2 *>(p);
#pragma unroll
    for (int j = 0; j < 3; ++j) q[j] = make_uint2(w[2 * j], w[2 * j + 1]);
  } else {
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int j = 0; j < CPL / 8; ++j) q[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
  }
}

// spilled first-direction costs: u8 when every real cost fits, else u16
template <int CPL, bool S8>
__device__ __forceinline__ void spill_put(uint8_t *p, const uint32_t (&w)[CPL / 2]) {
  if constexpr (S8)
    store_u8<CPL>(p, w);
  else
    store_u16<CPL>(reinterpret_cast<uint16_t *>(p), w);
}

template <int CPL, bool S8>
__device__ __forceinline__ void spill_get(const uint8_t *p, uint32_t (&w)[CPL / 2]) {
  if constexpr (S8) {
    const uint32_t z[CPL / 4] = {};
    unpack_u8<CPL>(p, z, w);
  } else {
    load_u16<CPL>(reinterpret_cast<const uint16_t *>(p), w);
  }
}

// ---- the recursion -----------------------------------------------------------
struct StepConsts {
  uint32_t p1x2;   // P1 in both halves
  uint32_t dpx2;   // (P2 - P1) in both halves
};

// One step of Eq. 2 for the lane's words.  mm = min_k L(p - r, k) in both
// halves; edge_lo / edge_hi are all-ones on the first / last lane of the
// group so that the missing neighbours L(-1) and L(Dp) read as 0xffff (they
// only enter a min).
// The step proper, given the word below the lane's first cell (prev: its
// high half is L(d-1) of the first cell) and the word above its last cell
// (next: its low half is L(d+1) of the last cell).
template <int NW>
__device__ __forceinline__ void sgm_core(uint32_t (&L)[NW], const uint32_t (&C)[NW], uint32_t mm,
                                         const StepConsts &sc, uint32_t prev, uint32_t next) {
  const uint32_t cap = mm + sc.dpx2;           // m + P2 - P1 per half
  const uint32_t negmm = 0u - mm;
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

template <int NW>
__device__ __forceinline__ void sgm_step(uint32_t (&L)[NW], const uint32_t (&C)[NW], uint32_t mm,
                                         const StepConsts &sc, uint32_t edge_lo, uint32_t edge_hi) {
  const uint32_t prev = __shfl_up_sync(kFull, L[NW - 1], 1, 16) | edge_lo;
  const uint32_t next = __shfl_down_sync(kFull, L[0], 1, 16) | edge_hi;
  sgm_core<NW>(L, C, mm, sc, prev, next);
}

// The step of the banded walks.  On the group's end lanes the missing
// neighbour is the lane's edge word e instead of all ones: lane 0 takes
// L(d-1) of its first cell from the high half of e, lane 15 L(d+1) of its
// last cell from the low half.  It is all ones (absent) except on the first
// step after a band change, where it holds the previous pixel's cell just
// outside the current band (band_shift).
template <int NW>
__device__ __forceinline__ void sgm_step_e(uint32_t (&L)[NW], const uint32_t (&C)[NW], uint32_t mm,
                                           const StepConsts &sc, uint32_t e, int lig) {
  const uint32_t up = __shfl_up_sync(kFull, L[NW - 1], 1, 16);
  const uint32_t dn = __shfl_down_sync(kFull, L[0], 1, 16);
  sgm_core<NW>(L, C, mm, sc, lig == 0 ? e : up, lig == 15 ? e : dn);
}

// Min of a u32 over each 16-lane group: two full-warp reductions, each with
// the other group's lanes contributing all-ones (a reduction over half a warp
// costs far more than two over the whole warp).
__device__ __forceinline__ uint32_t group_reduce_min(uint32_t v, int grp) {
  const uint32_t lo = __reduce_min_sync(kFull, grp ? 0xffffffffu : v);
  const uint32_t hi = __reduce_min_sync(kFull, grp ? v : 0xffffffffu);
  return grp ? hi : lo;
}

// min over the group's disparities, returned in both halves
template <int NW>
__device__ __forceinline__ uint32_t group_min(const uint32_t (&L)[NW], int grp) {
  uint32_t v = L[0];
#pragma unroll
  for (int i = 1; i + 1 < NW; i += 2) v = __vimin3_u16x2(v, L[i], L[i + 1]);
  if constexpr (NW % 2 == 0) v = __vminu2(v, L[NW - 1]);
  v = __vminu2(v, prmt(v, v, 0x1032));
  return group_reduce_min(v, grp);
}

// pad bytes (0x40 = high byte of kInf) of the lane's cells d >= D
template <int CPL>
__device__ __forceinline__ void pad_bytes(int D, int lig, uint32_t (&z)[CPL / 4]) {
#pragma unroll
  for (int i = 0; i < CPL / 4; ++i) {
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (lig * CPL + 4 * i + j >= D) v |= 0x40u << (8 * j);
    z[i] = v;
  }
}

// ---- disparity bands (banded mode, not in the paper) -----------------------------
// In banded mode lane cell j of pixel p stands for disparity lo_p + j, with
// lo_p constant on 8 x 8 pixel tiles.  A group walking its line tracks the
// tile of each step; where the band start changes by delta, the previous
// pixel's path costs are re-indexed: cell j takes old cell j + delta, and the
// cells that have no old counterpart become absent (kInf, above every real
// path cost, so they only ever lose a min).  m of the previous pixel stays
// the min over its own band.  The recursion on the bands is the exact
// dynamic program of Eq. 1 with each pixel's labels restricted to its band,
// so the previous pixel's cell just below the new band (old cell delta - 1,
// for delta > 0) or just above it (old cell B + delta, for delta < 0) is
// still the d-1 / d+1 neighbour of the new band's end cell: the shift hands
// it to the next step in the end lane's edge word.
struct BandState {
  const int16_t *lo = nullptr;   // this frame's tile table [th][tw]
  int tw = 0;
  int x = 0, y = 0;              // pixel of the next step
  int dx = 0, dy = 0;            // per-step move
  int tile = -1, cur = 0;        // tile and band start of the last step
  int kb_lo = -1;                // band start the row kernel's key bytes were built for
  uint16_t *buf = nullptr;       // the group's shared scratch, 16 * CPL cells
};

// Runs on all 32 lanes (full-warp syncs): a group with delta = 0 rewrites its
// cells in place.  Keeping the shift warp-uniform matters: the recursion's
// full-warp reductions must never meet a group parked at a partial barrier.
// edge receives the lane's edge word for the next step (sgm_step_e): on lane
// 0 the old cell delta - 1 in the high half, on lane 15 the old cell
// B + delta in the low half, all ones where that cell is outside the old band.
template <int CPL>
__device__ __forceinline__ void band_shift(uint32_t (&L)[CPL / 2], int delta, uint16_t *buf, int lig,
                                           uint32_t &edge) {
  constexpr int NW = CPL / 2, B = 16 * CPL;
  uint32_t *w = reinterpret_cast<uint32_t *>(buf + lig * CPL);
#pragma unroll
  for (int i = 0; i < NW; ++i) w[i] = L[i];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const int c0 = lig * CPL + 2 * i + delta;
    const uint32_t v0 = (unsigned)c0 < (unsigned)B ? (uint32_t)buf[c0] : kInf;
    const uint32_t v1 = (unsigned)(c0 + 1) < (unsigned)B ? (uint32_t)buf[c0 + 1] : kInf;
    L[i] = v0 | (v1 << 16);
  }
  const int ce = lig == 0 ? delta - 1 : B + delta;
  const uint32_t ve = (unsigned)ce < (unsigned)B ? (uint32_t)buf[ce] : 0xffffu;
  edge = lig == 0 ? (ve << 16) | 0xffffu : 0xffff0000u | ve;
  __syncwarp();
}

// the band bookkeeping of one step at (bs.x, bs.y), then the move to the next
// pixel of the line (x wraps for the diagonals).  Called by all 32 lanes;
// returns the change of the band start (0 for an inactive lane) and sets the
// lane's edge word for this step's recursion (all ones without a shift).
template <int CPL>
__device__ __forceinline__ int band_step(BandState &bs, uint32_t (&L)[CPL / 2], bool active, int W, int lig,
                                         uint32_t &edge) {
  int delta = 0;
  if (active) {
    const int t = (bs.y >> kBandTileLog) * bs.tw + (bs.x >> kBandTileLog);
    if (t != bs.tile) {
      bs.tile = t;
      const int nlo = bs.lo[t];
      delta = nlo - bs.cur;
      bs.cur = nlo;
    }
  }
  edge = 0xffffffffu;
  if (__any_sync(kFull, delta != 0)) band_shift<CPL>(L, delta, bs.buf, lig, edge);
  bs.y += bs.dy;
  bs.x += bs.dx;
  bs.x = bs.x >= W ? bs.x - W : (bs.x < 0 ? bs.x + W : bs.x);
  return delta;
}

// Banded right view.  At pixel x with band start lo, accumulator slot s holds
// the best key of right pixel x - lo - s.  From the previous pixel (x -/+ 1,
// band start lo - delta) slot s takes old slot s + sigma with sigma = delta - 1
// walking right and delta + 1 walking left; old slots that fall outside the
// band window are min-merged into merge[x'] (their right pixel may still get
// cells from pixels farther along, which merge there too).  Runs on all 32
// lanes through the group's shared buffer abuf (16 * CPL words).
template <int CPL>
__device__ __forceinline__ void band_acc_shift(uint32_t (&acc)[CPL], int sigma, int xr0, int W, uint32_t *abuf,
                                               uint32_t *merge, int lig) {
  constexpr int B = 16 * CPL;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int sl = lig * CPL + j;
    abuf[sl] = acc[j];
    const int to = sl - sigma;                     // the new slot of old slot sl
    if ((unsigned)to >= (unsigned)B && acc[j] != 0xffffffffu) {
      const int xr = xr0 - sl;                     // its right pixel
      if ((unsigned)xr < (unsigned)W) atomicMin(&merge[xr], acc[j]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int src = lig * CPL + j + sigma;
    acc[j] = (unsigned)src < (unsigned)B ? abuf[src] : 0xffffffffu;
  }
  __syncwarp();
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
  const int16_t *lo;      // banded mode: band starts per tile, [frame][th][tw]
  int tw, th;
  const int *gate;        // per-frame gate words of the launch's frames, or null
};

template <int CPL, bool S8, int NWARP>
struct LineCfg {
  static constexpr int Dp = 16 * CPL;
  static constexpr int K = CPL <= 8 ? 8 : 4;   // rows per stage
  static constexpr int S = 2;                  // stages per warp
  static constexpr int SB = S8 ? 1 : 2;        // spill bytes per cell
  static constexpr int kCost = K * 2 * Dp;     // [row][line of the warp][Dp]
  static constexpr int kSpillLine = K * Dp * SB;
  // S8: the up pass reads no spill (each pass writes its own byte plane)
  static constexpr int kStage = kCost + (S8 ? 0 : 2 * kSpillLine);
  static constexpr int kWarp = S * kStage;
  static constexpr int kWarps = NWARP;         // warps (two lines each) per CTA: a tuning choice
  static constexpr int kSmem = kWarps * kWarp + kWarps * S * 8;
};

// x of line k at row y in family fam
__device__ __forceinline__ int line_x(int fam, int k, int y, int W) {
  if (fam == 0) return k;
  int x = (fam == 1 ? k + y : k - y) % W;
  return x < 0 ? x + W : x;
}

// One chunk of n rows of a line walk (both lines of the warp).  DOWN: rows
// in increasing y, the path costs are spilled; up: rows in decreasing y, the
// spilled L_down of the row is added and the pair sum stored.  FAST: no path
// restarts inside the chunk (known from the warp-wide min of `togo`).
template <int CPL, bool S8, int FAM, bool DOWN, bool FAST, bool BANDED>
__device__ __forceinline__ void line_chunk(const uint8_t *stl, const uint8_t *sstl, int n, uint32_t (&L)[CPL / 2],
                                           uint32_t &mm, int &togo, int &next_len, int seg_full,
                                           uint8_t *&sp, uint8_t *&pp, const uint32_t (&z)[CPL / 4],
                                           const StepConsts &sc, uint32_t edge_lo, uint32_t edge_hi, int grp,
                                           bool active, int y_hi, int y_first, int W, uint8_t *part_lane,
                                           BandState &bs, int lig) {
  constexpr int NW = CPL / 2, Dp = 16 * CPL, SB = S8 ? 1 : 2;
  // The family buffer holds 2 Dp bytes per pixel: with S8 the down pass's
  // byte vector then the up pass's (pp walks this pass's half), otherwise the
  // u16 pair sum that the up pass forms from the down pass's spill (sp).
  constexpr int PS = 2 * Dp;
  // pixel pointer step per row: x - 1, x, x + 1 (families 1, 0, 2) going up,
  // the reverse going down
  constexpr int kDelta = FAM == 0 ? 0 : (FAM == 1 ? -1 : 1);
  const ptrdiff_t up_step = (ptrdiff_t)(kDelta - W) * PS;
  const ptrdiff_t down_step = (ptrdiff_t)(W - kDelta) * PS;
  uint32_t C[NW];
#pragma unroll 2
  for (int i = 0; i < n; ++i) {
    const int r = DOWN ? i : n - 1 - i;       // stage rows are in increasing y
    unpack_u8<CPL>(stl + r * 2 * Dp, z, C);
    uint32_t edge = 0xffffffffu;
    if (BANDED) band_step<CPL>(bs, L, active, W, lig, edge);
    if (!FAST) {
      const bool start = togo == 0;
      const uint32_t keep = start ? 0u : 0xffffffffu;
#pragma unroll
      for (int w = 0; w < NW; ++w) L[w] &= keep;
      mm &= keep;
      if (start) {
        togo = next_len;
        next_len = seg_full;
        // a diagonal line restarts (after its first pixel) where x wrapped
        // around: going up at x = W-1 for family 1, x = 0 for family 2;
        // going down at x = 0 for family 1, x = W-1 for family 2
        if (!DOWN && FAM != 0) {
          const int y = y_hi - i;
          if (y != y_first) pp = part_lane + (size_t)(y * W + (FAM == 1 ? W - 1 : 0)) * PS;
        }
        if (S8 && DOWN && FAM != 0) {
          const int y = y_hi - (n - 1) + i;
          if (y != 0) pp = part_lane + (size_t)(y * W + (FAM == 1 ? 0 : W - 1)) * PS;
        }
      }
      --togo;
    }
    if constexpr (BANDED)
      sgm_step_e<NW>(L, C, mm, sc, edge, lig);
    else
      sgm_step<NW>(L, C, mm, sc, edge_lo, edge_hi);
    mm = group_min<NW>(L, grp);
    if constexpr (S8) {
      // this direction's path costs, one byte per cell, in its half of the pixel's slot
      if (active) store_u8<CPL>(pp, L);
      pp += DOWN ? down_step : up_step;
    } else if (DOWN) {
      if (active) spill_put<CPL, S8>(sp, L);
      sp += Dp * SB;
    } else {
      uint32_t Ld[NW];
      spill_get<CPL, S8>(sstl + r * Dp * SB, Ld);
#pragma unroll
      for (int w = 0; w < NW; ++w) Ld[w] += L[w];
      if (active) store_u16<CPL>(reinterpret_cast<uint16_t *>(pp), Ld);
      pp += up_step;
    }
  }
  if (FAST) togo -= n;
}

template <int CPL, bool S8, int FAM, int NWARP, bool BANDED>
__global__ void __launch_bounds__(32 * NWARP) k_agg_lines(const __grid_constant__ LineArgs a) {
  using CF = LineCfg<CPL, S8, NWARP>;
  constexpr int NW = CPL / 2, K = CF::K, S = CF::S, Dp = CF::Dp, SB = CF::SB;
  extern __shared__ __align__(128) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> 4, lig = lane & 15;
  const int f = blockIdx.y;
  if (gated_off(a.gate ? a.gate + f : nullptr, a.k.gate_run)) return;
  const int W = a.k.W, H = a.k.H;
  const size_t fcells = frame_cells(a.k);
  const uint8_t *cost = a.cost + f * fcells;
  // the family's buffer of this frame, 2 Dp bytes per pixel: [L_down][L_up]
  // bytes for S8, else the u16 pair sums
  uint8_t *part = reinterpret_cast<uint8_t *>(a.part[FAM] + f * fcells);
  const int line0 = (blockIdx.x * CF::kWarps + warp) * 2;
  if (line0 >= W) return;                    // warps are independent: no block barrier below
  const int line = line0 + grp;
  const bool active = line < W;              // the second group of the last warp may idle
  const int nact = line0 + 1 < W ? 2 : 1;
  uint8_t *ring = smem + warp * CF::kWarp;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + CF::kWarps * CF::kWarp) + warp * S;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  uint32_t z[CPL / 4];
  pad_bytes<CPL>(a.k.D, lig, z);
  const uint32_t edge_lo = lig == 0 ? 0xffffffffu : 0u, edge_hi = lig == 15 ? 0xffffffffu : 0u;
  const StepConsts sc = a.sc;
  uint8_t *spill = static_cast<uint8_t *>(a.spill) + f * 4 * fcells * 2;   // this frame's spill regions
  const size_t spill0 = ((size_t)FAM * W + line0) * (size_t)H * Dp;     // elements, line0
  const size_t spill_line = spill0 + (size_t)grp * H * Dp;
  const int nch = (H + K - 1) / K;
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
    if (lane == 0) mbar_expect_tx(&bars[stage], (uint32_t)(nact * n * Dp * (up && !S8 ? 1 + SB : 1)));
    __syncwarp();
    const int r = lane >> 1, gg = lane & 1;
    if (r < n && line0 + gg < W) {
      const int y = y_lo + r;
      bulk_g2s(st + (r * 2 + gg) * Dp, cost + ((size_t)y * W + line_x(FAM, line0 + gg, y, W)) * Dp, Dp,
               &bars[stage]);
    }
    if (!S8 && up && lane >= 30 && line0 + (lane - 30) < W) {
      const int l = lane - 30;
      bulk_g2s(st + CF::kCost + l * CF::kSpillLine,
               spill + (spill0 + (size_t)l * H * Dp + (size_t)y_lo * Dp) * SB, (uint32_t)(n * Dp * SB),
               &bars[stage]);
    }
  };

  uint32_t L[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) L[w] = 0;
  uint32_t mm = 0;
  // Path restarts: togo = steps until the next restart (0: this step restarts).
  const int x_top = line_x(FAM, line, 0, W), x_bot = line_x(FAM, line, H - 1, W);
  const int seg_full = FAM == 0 ? 0x7fffffff : W;
  const int cost_off = grp * Dp + lig * CPL;                          // lane's cells in a stage row
  const int spill_off = CF::kCost + grp * CF::kSpillLine + lig * CPL * SB;
  // banded mode: the group's shift scratch follows the barriers
  BandState bs;
  if (BANDED) {
    bs.lo = a.lo + (size_t)f * a.th * a.tw;
    bs.tw = a.tw;
    bs.buf = reinterpret_cast<uint16_t *>(smem + CF::kSmem) + (warp * 2 + grp) * Dp;
    bs.x = x_top;
    bs.y = 0;
    bs.dy = 1;
    bs.dx = FAM == 0 ? 0 : (FAM == 1 ? 1 : -1);
  }
  // ---- down: r = (0,1), (1,1), (-1,1) ----
  int togo = 0;
  int next_len = FAM == 0 ? 0x7fffffff : (FAM == 1 ? W - x_top : x_top + 1);
  {
    uint8_t *sp = spill + (spill_line + (size_t)lig * CPL) * SB;
    uint8_t *down_lane = part + lig * CPL;                                  // S8: the down half
    uint8_t *pp = S8 ? down_lane + (size_t)x_top * 2 * Dp : nullptr;
    int issued = 0;
    for (int c = 0; c < nch; ++c) {
      while (issued < nch && issued < c + S) issue(issued++);
      if (!ring_wait<S>(bars, c, issued, a.err)) return;
      const int n = min(K, H - c * K);
      const uint8_t *st = ring + (c % S) * CF::kStage;
      const bool fast = __reduce_min_sync(kFull, (unsigned)(active ? togo : 0x7fffffff)) >= (unsigned)n;
      if (fast)
        line_chunk<CPL, S8, FAM, true, true, BANDED>(st + cost_off, st + spill_off, n, L, mm, togo, next_len,
                                                     seg_full, sp, pp, z, sc, edge_lo, edge_hi, grp, active,
                                                     c * K + n - 1, H - 1, W, down_lane, bs, lig);
      else
        line_chunk<CPL, S8, FAM, true, false, BANDED>(st + cost_off, st + spill_off, n, L, mm, togo, next_len,
                                                      seg_full, sp, pp, z, sc, edge_lo, edge_hi, grp, active,
                                                      c * K + n - 1, H - 1, W, down_lane, bs, lig);
      __syncwarp();
    }
  }
  // the spilled L_down rows are read back by bulk copies (async proxy)
  fence_proxy_async_global();
  __syncwarp();
  // ---- up: r = (0,-1), (-1,-1), (1,-1); emit L_down + L_up ----
  togo = 0;
  next_len = FAM == 0 ? 0x7fffffff : (FAM == 1 ? x_bot + 1 : W - x_bot);
  if (BANDED) {
    bs.x = x_bot;
    bs.y = H - 1;
    bs.dy = -1;
    bs.dx = FAM == 0 ? 0 : (FAM == 1 ? -1 : 1);
    bs.tile = -1;          // the up walk starts afresh (its first step restarts the path)
  }
  {
    uint8_t *sp = nullptr;
    uint8_t *part_lane = S8 ? part + Dp + lig * CPL : part + lig * CPL * 2;   // S8: the up half
    uint8_t *pp = part_lane + (size_t)((H - 1) * W + x_bot) * 2 * Dp;
    int issued = nch;
    for (int c = 0; c < nch; ++c) {
      const int g = nch + c;
      while (issued < 2 * nch && issued < g + S) issue(issued++);
      if (!ring_wait<S>(bars, g, issued, a.err)) return;
      const int y_hi = H - 1 - c * K, n = y_hi - max(0, y_hi - K + 1) + 1;
      const uint8_t *st = ring + (g % S) * CF::kStage;
      const bool fast = __reduce_min_sync(kFull, (unsigned)(active ? togo : 0x7fffffff)) >= (unsigned)n;
      if (fast)
        line_chunk<CPL, S8, FAM, false, true, BANDED>(st + cost_off, st + spill_off, n, L, mm, togo, next_len,
                                                      seg_full, sp, pp, z, sc, edge_lo, edge_hi, grp, active, y_hi,
                                                      H - 1, W, part_lane, bs, lig);
      else
        line_chunk<CPL, S8, FAM, false, false, BANDED>(st + cost_off, st + spill_off, n, L, mm, togo, next_len,
                                                       seg_full, sp, pp, z, sc, edge_lo, edge_hi, grp, active, y_hi,
                                                       H - 1, W, part_lane, bs, lig);
      __syncwarp();
    }
  }
}

// ---- rows, path sum and WTA ----------------------------------------------------
// One warp per image row.  Group 0 walks left -> right (r = (1,0)), group 1
// right -> left (r = (-1,0)), in lockstep.  Each group spills its path costs
// for the half of the row it reaches first (group 0: x < xm, group 1:
// x >= xm); on the half it reaches second it reads the other group's spill,
// adds the line-family sums into S, and takes d* and d' there.  For odd W
// group 0 starts one step late so that both first halves end together.  The
// right-view keys of pixels x' whose diagonal crosses xm are merged in shared
// memory at the end.
struct RowArgs {
  KParams k;
  const uint8_t *cost;
  const uint16_t *part[3];
  void *spill;            // frame 0 spill regions; the row region is the fourth
  int16_t *dstar, *dprime;
  int16_t *dsub;          // sub-pixel output (1/16 px), or null when the fit is off
  uint16_t *dbg_sum;
  int *err;
  StepConsts sc;
  const int16_t *lo;      // banded mode: band starts per tile, [frame][th][tw]
  int tw, th;
  const int *gate;        // per-frame gate words of the launch's frames, or null
};

template <int CPL, bool S8, int NP>
struct RowCfg {
  static constexpr int Dp = 16 * CPL;
  static constexpr int K = CPL <= 8 ? 4 : 2;    // walk steps per stage
  static constexpr int S = 2;
  static constexpr int SB = S8 ? 1 : 2;
  static constexpr int kCost = K * Dp;
  static constexpr int kSpill = K * Dp * SB;
  static constexpr int kPart = K * Dp * 2;
  static constexpr int kGroup = kCost + kSpill + NP * kPart;  // per group and stage: one slot per family buffer
  static constexpr int kStage = 2 * kGroup;
  static constexpr int kSmem = S * kStage + S * 8 + kMaxDisp * 4;
};

// per-warp state of the row walk
template <int CPL>
struct RowWalk {
  uint32_t L[CPL / 2];
  uint32_t mm;
  uint32_t acc[CPL];      // right-view keys; slot d holds right pixel x - d
};

struct RowGeom {
  int W, D, xm, delay, mbase, lastLig, lastSlot;
  bool fwd;
  size_t row;
};

// one chunk of lockstep steps [t_lo, t_hi); SECOND: the half where S is formed;
// RESTART: the chunk holds the first step of a walk
template <int CPL, bool S8, int NP, bool FULLD, bool SECOND, bool RESTART, bool BANDED, bool FULL>
__device__ __forceinline__ void row_chunk(RowWalk<CPL> &w, const RowGeom &g, const uint8_t *stg, int xl, int t_lo,
                                          int t_hi, const uint32_t (&z)[CPL / 4], uint32_t (&kb)[CPL / 2],
                                          const StepConsts &sc, uint32_t edge_lo, uint32_t edge_hi, int grp, int lig,
                                          uint8_t *spill_lane, int16_t *dstar, int16_t *dprime, int16_t *dsub,
                                          uint16_t *dbg_lane, uint32_t *merge, BandState &bs, uint32_t *abuf) {
  using CF = RowCfg<CPL, S8, NP>;
  constexpr int NW = CPL / 2, Dp = CF::Dp, SB = CF::SB;
  const uint8_t *cst = stg + lig * CPL;
  const uint8_t *sst = stg + CF::kCost + lig * CPL * SB;
  // family sums, 2 Dp bytes per pixel: u16 pair sums, or (S8) the down and
  // up passes' byte vectors; NP == 2: the down and up sweeps' u16 sums of
  // three directions each
  constexpr bool kPartBytes = S8 && NP != 2;   // byte vectors, else u16 sums
  const uint8_t *pst = stg + CF::kCost + CF::kSpill + lig * CPL * (kPartBytes ? 1 : 2);
  // one step at t; FULL: a chunk of K steps whose pixels are all in the
  // image (both groups), unrolled
  auto step_at = [&](const int t) {
    const int x = g.fwd ? t - g.delay : g.W - 1 - t;
    const bool valid = FULL || (x >= 0 && x < g.W);
    const int r = valid ? x - xl : 0;
    uint32_t C[NW];
    unpack_u8<CPL>(cst + r * Dp, z, C);
    int delta = 0;
    uint32_t edge = 0xffffffffu;
    if (BANDED) {
      bs.x = x;   // rows: the tile follows x (bs.y is the row)
      delta = band_step<CPL>(bs, w.L, valid, g.W, lig, edge);
      if (SECOND && bs.cur != bs.kb_lo) {
        // keys carry absolute disparities: lo + slot
        bs.kb_lo = bs.cur;
        const uint32_t b0 = (uint32_t)(bs.cur + lig * CPL);
#pragma unroll
        for (int i = 0; i < CPL / 2; ++i) kb[i] = (b0 + 2 * i) | ((b0 + 2 * i + 1) << 8);
      }
    }
    if (RESTART) {
      // a walk starts at x = 0 (group 0) / x = W-1 (group 1): zero previous vector
      const uint32_t keep = x == (g.fwd ? 0 : g.W - 1) ? 0u : 0xffffffffu;
#pragma unroll
      for (int i = 0; i < NW; ++i) w.L[i] &= keep;
      w.mm &= keep;
    }
    if constexpr (BANDED)
      sgm_step_e<NW>(w.L, C, w.mm, sc, edge, lig);
    else
      sgm_step<NW>(w.L, C, w.mm, sc, edge_lo, edge_hi);
    w.mm = group_min<NW>(w.L, grp);
    if (!SECOND) {
      if (valid) spill_put<CPL, S8>(spill_lane + (size_t)x * Dp * SB, w.L);
      return;
    }
    uint32_t Sm[NW];
    spill_get<CPL, S8>(sst + r * Dp * SB, Sm);
#pragma unroll
    for (int i = 0; i < NW; ++i) Sm[i] += w.L[i];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      uint32_t T[NW];
      if constexpr (kPartBytes) {
        const uint32_t z0[CPL / 4] = {};
        uint32_t U[NW];
        unpack_u8<CPL>(pst + j * CF::kPart + r * 2 * Dp, z0, T);         // L_down of the family
        unpack_u8<CPL>(pst + j * CF::kPart + r * 2 * Dp + Dp, z0, U);    // L_up
#pragma unroll
        for (int i = 0; i < NW; ++i) T[i] += U[i];
      } else {
        load_u16<CPL>(reinterpret_cast<const uint16_t *>(pst + j * CF::kPart + r * Dp * 2), T);
      }
#pragma unroll
      for (int i = 0; i < NW; ++i) Sm[i] += T[i];
    }
    if (dbg_lane != nullptr && valid) store_u16<CPL>(dbg_lane + (size_t)x * Dp, Sm);
    // keys (S << 8 | d); padding keys have 0xff in the top byte
    uint32_t key[CPL];
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      key[2 * i] = prmt(Sm[i], kb[i], 0x6104);
      key[2 * i + 1] = prmt(Sm[i], kb[i], 0x7325);
    }
    uint32_t best = key[0];
#pragma unroll
    for (int j = 1; j < CPL; ++j) best = min(best, key[j]);
    best = group_reduce_min(best, grp);
    if (lig == 0 && valid) dstar[g.row + x] = (int16_t)(best & 0xffu);
    if (dsub != nullptr) {
      // parabola through S(d*-1), S(d*), S(d*+1); the lanes holding the two
      // neighbours contribute them, every other lane the neutral 0xffffffff
      const int ds = (int)(best & 0xffu);
      uint32_t sm = 0xffffffffu, sp = 0xffffffffu;
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int d = lig * CPL + j;
        sm = d + 1 == ds ? key[j] >> 8 : sm;
        sp = d == ds + 1 ? key[j] >> 8 : sp;
      }
      sm = group_reduce_min(sm, grp);
      sp = group_reduce_min(sp, grp);
      if (lig == 0 && valid) {
        int v = 16 * ds;
        if (ds > 0 && ds < g.D - 1) {
          // d* is the smallest argmin: den = S(d*-1) - 2 S(d*) + S(d*+1) > 0 and
          // 16 (S(d*-1) - S(d*+1)) > -16 den, so the biased numerator is positive:
          // offset = floor((16 (sm - sp) + den) / (2 den)) = that quotient - 8
          const uint32_t s0 = best >> 8, den = sm + sp - 2u * s0;
          v += (int)((16u * sm + 17u * den - 16u * sp) / (2u * den)) - 8;
        }
        dsub[g.row + x] = (int16_t)v;
      }
    }
    if (BANDED) {
      // right view on the bands: re-index the accumulator to this pixel's
      // window (emitting the slots that leave it), then fold in S(x, d)
      const int xr0 = (g.fwd ? x - 1 : x + 1) - (bs.cur - delta);   // right pixel of old slot 0
      if (__any_sync(kFull, delta != 0)) {
        const int sigma = g.fwd ? delta - 1 : delta + 1;
        band_acc_shift<CPL>(w.acc, valid ? sigma : 0, valid ? xr0 : -0x40000000, g.W, abuf, merge, lig);
        if (valid) {
#pragma unroll
          for (int j = 0; j < CPL; ++j) w.acc[j] = min(w.acc[j], key[j]);
        }
      } else {
        // same band as the previous pixel: the plain one-slot move, and the
        // slot that leaves the window goes to the merge array
        const uint32_t sh_up = __shfl_up_sync(kFull, w.acc[CPL - 1], 1, 16);
        const uint32_t sh_dn = __shfl_down_sync(kFull, w.acc[0], 1, 16);
        if (valid) {
          const int eslot = g.fwd ? 16 * CPL - 1 : 0;
          const uint32_t out = g.fwd ? w.acc[CPL - 1] : w.acc[0];
          if (lig == (g.fwd ? 15 : 0) && out != 0xffffffffu && (unsigned)(xr0 - eslot) < (unsigned)g.W)
            atomicMin(&merge[xr0 - eslot], out);
          const uint32_t in_up = lig == 0 ? 0xffffffffu : sh_up;
          const uint32_t in_dn = lig == 15 ? 0xffffffffu : sh_dn;
          uint32_t nacc[CPL];
#pragma unroll
          for (int j = 0; j < CPL; ++j) {
            const uint32_t lower = j == 0 ? in_up : w.acc[j - 1];
            const uint32_t upper = j == CPL - 1 ? in_dn : w.acc[j + 1];
            nacc[j] = min(g.fwd ? lower : upper, key[j]);
          }
#pragma unroll
          for (int j = 0; j < CPL; ++j) w.acc[j] = nacc[j];
        }
      }
      return;
    }
    // right view: group 0 (x rising) moves keys up a slot per step, group 1
    // (x falling) down a slot; both fold in S(x, d)
    // (shuffles run on every lane: the full-warp mask requires it)
    const uint32_t sh_up = __shfl_up_sync(kFull, w.acc[CPL - 1], 1, 16);
    const uint32_t sh_dn = __shfl_down_sync(kFull, w.acc[0], 1, 16);
    const uint32_t in_up = lig == 0 ? 0xffffffffu : sh_up;
    const uint32_t in_dn = lig == 15 ? 0xffffffffu : sh_dn;
    if (valid) {
      uint32_t nacc[CPL];
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const uint32_t lower = j == 0 ? in_up : w.acc[j - 1];
        const uint32_t upper = j == CPL - 1 ? in_dn : w.acc[j + 1];
        nacc[j] = min(g.fwd ? lower : upper, key[j]);
      }
#pragma unroll
      for (int j = 0; j < CPL; ++j) w.acc[j] = nacc[j];
      const int elane = g.fwd ? g.lastLig : 0;
      const int xr = g.fwd ? x - (g.D - 1) : x;
      if (lig == elane && xr >= 0) {
        uint32_t v = w.acc[0];
        if (g.fwd) {
          if (FULLD) {
            v = w.acc[CPL - 1];
          } else {
#pragma unroll
            for (int j = 1; j < CPL; ++j)
              if (j == g.lastSlot) v = w.acc[j];
          }
        }
        const bool fin = g.fwd ? xr >= g.xm : x + g.D - 1 < g.xm;
        if (fin)
          dprime[g.row + xr] = (int16_t)(v & 0xffu);
        else
          atomicMin(&merge[xr - g.mbase], v);
      }
    }
  };
  if constexpr (FULL) {
#pragma unroll
    for (int u = 0; u < CF::K; ++u) step_at(t_lo + u);
  } else {
    for (int t = t_lo; t < t_hi; ++t) step_at(t);
  }
}

template <int CPL, bool S8, int NP, bool FULLD, bool BANDED>
__global__ void __launch_bounds__(32) k_agg_rows(const __grid_constant__ RowArgs a) {
  using CF = RowCfg<CPL, S8, NP>;
  constexpr int K = CF::K, S = CF::S, Dp = CF::Dp, SB = CF::SB;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S * CF::kStage);
  uint32_t *merge = reinterpret_cast<uint32_t *>(smem + S * CF::kStage + S * 8);
  const int lane = threadIdx.x & 31, grp = lane >> 4, lig = lane & 15;
  const int y = blockIdx.x, f = blockIdx.y;
  if (gated_off(a.gate ? a.gate + f : nullptr, a.k.gate_run)) return;
  RowGeom g;
  g.W = a.k.W;
  g.D = a.k.D;
  g.fwd = grp == 0;
  g.xm = g.W / 2;
  g.delay = g.W & 1;                       // group 0 idles in step 0 when W is odd
  g.mbase = g.xm - g.D + 1;                // merge slot i holds right pixel mbase + i
  g.lastLig = (g.D - 1) / CPL;
  g.lastSlot = (g.D - 1) % CPL;
  g.row = (size_t)y * g.W;
  const int W = g.W, D = g.D;
  const size_t fcells = frame_cells(a.k), fpx = frame_px(a.k);
  const uint8_t *cost = a.cost + f * fcells;
  const uint16_t *part0 = a.part[0] + f * fcells, *part1 = a.part[1] + f * fcells, *part2 = a.part[2] + f * fcells;
  int16_t *dstar = a.dstar + f * fpx, *dprime = a.dprime + f * fpx;
  int16_t *dsub = a.dsub != nullptr ? a.dsub + f * fpx : nullptr;
  uint16_t *dbg_lane = (f == 0 && a.dbg_sum != nullptr) ? a.dbg_sum + g.row * Dp + lig * CPL : nullptr;
  BandState bs;
  uint32_t *abuf = nullptr;
  if (BANDED) {
    // shared memory after the merge array (one word per right pixel of the
    // row): each group's path-cost shift buffer, then its accumulator buffer
    bs.lo = a.lo + (size_t)f * a.th * a.tw;
    bs.tw = a.tw;
    bs.y = y;
    uint16_t *lbuf = reinterpret_cast<uint16_t *>(merge + W);
    bs.buf = lbuf + grp * Dp;
    abuf = reinterpret_cast<uint32_t *>(lbuf + 2 * Dp) + grp * Dp;
  }
  // the row spill region of this frame
  uint8_t *spill = static_cast<uint8_t *>(a.spill) + f * 4 * fcells * 2 + 3 * fcells * SB;
  uint8_t *spill_lane = spill + (g.row * Dp + lig * CPL) * SB;
  const int tmid = g.xm + g.delay;         // both first halves end here
  const int T = W + g.delay;               // lockstep steps
  const int c1 = (tmid + K - 1) / K, c2 = (T - tmid + K - 1) / K, nch = c1 + c2;
  for (int i = lane; i < (BANDED ? W : kMaxDisp); i += 32) merge[i] = 0xffffffffu;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncwarp();
  uint32_t z[CPL / 4];
  pad_bytes<CPL>(D, lig, z);
  const uint32_t edge_lo = lig == 0 ? 0xffffffffu : 0u, edge_hi = lig == 15 ? 0xffffffffu : 0u;
  const StepConsts sc = a.sc;
  uint32_t kb[CPL / 2];
#pragma unroll
  for (int i = 0; i < CPL / 2; ++i) {
    const int d0 = lig * CPL + 2 * i;
    kb[i] = (uint32_t)(d0 & 0xff) | ((uint32_t)((d0 + 1) & 0xff) << 8) | (d0 >= D ? 0xff0000u : 0u) |
            (d0 + 1 >= D ? 0xff000000u : 0u);
  }
  auto chunk = [&](int c, int &t_lo, int &t_hi) {
    if (c < c1) {
      t_lo = c * K;
      t_hi = min(tmid, t_lo + K);
    } else {
      t_lo = tmid + (c - c1) * K;
      t_hi = min(T, t_lo + K);
    }
  };
  // pixels of group gg in steps [t_lo, t_hi): [x_lo, x_lo + n)
  auto span = [&](int gg, int t_lo, int t_hi, int &x_lo, int &n) {
    int a0 = gg == 0 ? t_lo - g.delay : W - t_hi;
    int a1 = gg == 0 ? t_hi - 1 - g.delay : W - 1 - t_lo;
    a0 = max(a0, 0);
    a1 = min(a1, W - 1);
    x_lo = a0;
    n = a1 >= a0 ? a1 - a0 + 1 : 0;
  };
  auto issue = [&](int c) {
    int t_lo, t_hi;
    chunk(c, t_lo, t_hi);
    const bool second = c >= c1;
    const int stage = c % S;
    int xl0, nn0, xl1, nn1;
    span(0, t_lo, t_hi, xl0, nn0);
    span(1, t_lo, t_hi, xl1, nn1);
    const uint32_t per_px = (uint32_t)(Dp * (second ? 1 + SB + 2 * NP : 1));
    if (lane == 0) mbar_expect_tx(&bars[stage], (uint32_t)(nn0 + nn1) * per_px);
    __syncwarp();
    // lanes 0..4 serve group 0, lanes 16..20 group 1: cost, other group's spill, parts
    const int xl = grp ? xl1 : xl0, nn = grp ? nn1 : nn0, j = lig;
    if (nn > 0) {
      uint8_t *st = smem + stage * CF::kStage + grp * CF::kGroup;
      const size_t cell = (g.row + xl) * Dp;
      if (j == 0) bulk_g2s(st, cost + cell, (uint32_t)(nn * Dp), &bars[stage]);
      if (second) {
        if (j == 1) bulk_g2s(st + CF::kCost, spill + cell * SB, (uint32_t)(nn * Dp * SB), &bars[stage]);
        if (j >= 2 && j < 2 + NP)   // 2 Dp bytes per pixel in either layout
          bulk_g2s(st + CF::kCost + CF::kSpill + (j - 2) * CF::kPart,
                   (j == 2 ? part0 : (j == 3 ? part1 : part2)) + cell, (uint32_t)(nn * Dp * 2), &bars[stage]);
      }
    }
  };
  RowWalk<CPL> w;
#pragma unroll
  for (int i = 0; i < CPL / 2; ++i) w.L[i] = 0;
  w.mm = 0;
#pragma unroll
  for (int j = 0; j < CPL; ++j) w.acc[j] = 0xffffffffu;
  bool ok = true;
  int issued = 0;
  for (int c = 0; c < nch; ++c) {
    // second-half fills read the other group's spill: issue them only after
    // both first halves are stored and fenced (end of chunk c1 - 1)
    while (issued < nch && issued < c + S && (issued < c1 || c >= c1)) issue(issued++);
    if (!ring_wait<S>(bars, c, issued, a.err)) {
      ok = false;
      break;
    }
    int t_lo, t_hi;
    chunk(c, t_lo, t_hi);
    int xl, nn;
    span(grp, t_lo, t_hi, xl, nn);
    const uint8_t *stg = smem + (c % S) * CF::kStage + grp * CF::kGroup;
    // a walk starts at step delay (group 0) or 0 (group 1)
    const bool restart = t_lo <= g.delay && 0 < t_hi;
#define ROW_CHUNK(SEC, RS, FU)                                                                               \
  row_chunk<CPL, S8, NP, FULLD, SEC, RS, BANDED, FU>(w, g, stg, xl, t_lo, t_hi, z, kb, sc, edge_lo, edge_hi, grp, \
                                                     lig, spill_lane, dstar, dprime, dsub, dbg_lane, merge, bs, abuf)
    // a full chunk: K steps, every pixel of both groups in the image
    constexpr bool kFullChunks = true;
    const bool full = kFullChunks && !restart && t_hi - t_lo == K && t_lo >= g.delay &&
                      t_hi - 1 - g.delay < W && t_hi - 1 < W;
    if (c < c1) {
      if (restart)
        ROW_CHUNK(false, true, false);
      else if (full)
        ROW_CHUNK(false, false, true);
      else
        ROW_CHUNK(false, false, false);
    } else {
      if (restart)
        ROW_CHUNK(true, true, false);
      else if (full)
        ROW_CHUNK(true, false, true);
      else
        ROW_CHUNK(true, false, false);
    }
#undef ROW_CHUNK
    __syncwarp();
    if (c + 1 == c1) {
      // both groups' first halves are stored: make them visible to the bulk copies
      fence_proxy_async_global();
      __syncwarp();
    }
  }
  if (BANDED) {
    if (ok) {
      // the slots still held at the end of each walk, then d' of every right
      // pixel from the merged keys (-1 where no band holds a cell of its diagonal)
      const int xr0 = (g.fwd ? W - 1 : 0) - bs.cur;
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const int xr = xr0 - (lig * CPL + j);
        if (w.acc[j] != 0xffffffffu && (unsigned)xr < (unsigned)W) atomicMin(&merge[xr], w.acc[j]);
      }
      __syncwarp();
      for (int i = lane; i < W; i += 32)
        dprime[g.row + i] = merge[i] == 0xffffffffu ? (int16_t)-1 : (int16_t)(merge[i] & 0xffu);
    }
    return;
  }
  if (ok && g.fwd) {
    // right pixels x' = W-1-d whose diagonal leaves the image: slot d of group 0
#pragma unroll
    for (int j = 0; j < CPL; ++j) {
      const int d = lig * CPL + j, xr = W - 1 - d;
      if (d < D - 1 && xr >= 0) {
        if (xr >= g.xm)
          dprime[g.row + xr] = (int16_t)(w.acc[j] & 0xffu);
        else
          atomicMin(&merge[xr - g.mbase], w.acc[j]);
      }
    }
  }
  __syncwarp();
  if (ok) {
    // right pixels whose diagonal crosses xm: both groups contributed
    for (int i = lane; i < D - 1; i += 32) {
      const int xr = g.mbase + i;
      if (xr >= 0 && xr < g.xm) dprime[g.row + xr] = (int16_t)(merge[i] & 0xffu);
    }
  }
}

// opt in once per device to the kernel's dynamic shared memory
template <typename Kern>
static cudaError_t smem_optin(Kern kern, int bytes, bool (&done)[64]) {
  return once_per_device(done, [&](int) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  });
}

template <int CPL, bool S8, int FAM, int NWARP, bool BANDED>
static cudaError_t launch_line_family_w(const LineArgs &a, int nf, cudaStream_t s) {
  using CF = LineCfg<CPL, S8, NWARP>;
  constexpr int kSmem = CF::kSmem + (BANDED ? CF::kWarps * 4 * CF::Dp : 0);   // + shift scratch
  static bool done[64] = {};
  cudaError_t e = smem_optin(k_agg_lines<CPL, S8, FAM, NWARP, BANDED>, kSmem, done);
  if (e != cudaSuccess) return e;
  const int lines_per_cta = 2 * CF::kWarps;
  dim3 grid((a.k.W + lines_per_cta - 1) / lines_per_cta, nf);
  k_agg_lines<CPL, S8, FAM, NWARP, BANDED><<<grid, 32 * CF::kWarps, kSmem, s>>>(a);
  return cudaGetLastError();
}

// warps per CTA from the context's tuning (1, 2, 4 or 8); the banded variant
// exists for 4 warps and up to 8 cells per lane (bands of 64 or 128)
template <int CPL, bool S8, int FAM>
static cudaError_t launch_line_family(const LineArgs &a, int nf, cudaStream_t s) {
  if (a.lo != nullptr) {
    if constexpr (CPL <= 8) return launch_line_family_w<CPL, S8, FAM, 4, true>(a, nf, s);
    return cudaErrorInvalidValue;
  }
  switch (a.k.line_warps) {
    case 1: return launch_line_family_w<CPL, S8, FAM, 1, false>(a, nf, s);
    case 2: return launch_line_family_w<CPL, S8, FAM, 2, false>(a, nf, s);
    case 8: return launch_line_family_w<CPL, S8, FAM, 8, false>(a, nf, s);
    default: return launch_line_family_w<CPL, S8, FAM, 4, false>(a, nf, s);
  }
}

// In banded mode (k.band != 0) the kernels see D = Dp = band: lane cells are
// band positions, never padding.
static KParams lane_params(const KParams &k) {
  KParams kk = k;
  if (k.band) kk.D = k.Dp;
  return kk;
}

template <int CPL, bool S8>
cudaError_t launch_lines_t(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  LineArgs a;
  a.k = lane_params(k);
  a.cost = b.cost;
  for (int i = 0; i < 3; ++i) a.part[i] = b.part[i];
  a.spill = b.spill;
  a.err = b.err;
  a.sc.p1x2 = (uint32_t)k.p1 * 0x10001u;
  a.sc.dpx2 = (uint32_t)(k.p2 - k.p1) * 0x10001u;
  a.lo = k.band ? b.band_lo : nullptr;
  a.tw = k.tw;
  a.th = k.th;
  a.gate = b.gate;
  // the three families are independent: one launch each, back to back
  cudaError_t e = launch_line_family<CPL, S8, 0>(a, nf, s);
  if (e != cudaSuccess || k.num_paths != 8) return e;
  e = launch_line_family<CPL, S8, 1>(a, nf, s);
  if (e != cudaSuccess) return e;
  return launch_line_family<CPL, S8, 2>(a, nf, s);
}

template <int CPL, bool S8, int NP, bool FULLD, bool BANDED>
static cudaError_t launch_rows_v(const RowArgs &a, int nf, cudaStream_t s) {
  using CF = RowCfg<CPL, S8, NP>;
  // banded: the merge array grows to one word per pixel of the row, followed
  // by the two groups' shift buffers (u16 path costs, u32 accumulators)
  constexpr int kBandMax = CF::kSmem - kMaxDisp * 4 + kMaxDim * 4 + 2 * CF::Dp * 2 + 2 * CF::Dp * 4;
  const int smem = BANDED ? CF::kSmem - kMaxDisp * 4 + a.k.W * 4 + 2 * CF::Dp * 2 + 2 * CF::Dp * 4 : CF::kSmem;
  static bool done[64] = {};
  cudaError_t e = smem_optin(k_agg_rows<CPL, S8, NP, FULLD, BANDED>, BANDED ? kBandMax : CF::kSmem, done);
  if (e != cudaSuccess) return e;
  k_agg_rows<CPL, S8, NP, FULLD, BANDED><<<dim3(a.k.H, nf), 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int CPL, bool S8>
cudaError_t launch_rows_t(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  RowArgs a;
  a.k = lane_params(k);
  a.cost = b.cost;
  for (int i = 0; i < 3; ++i) a.part[i] = b.part[i];
  a.spill = b.spill;
  a.dstar = b.dstar;
  a.dprime = b.dprime;
  a.dsub = k.subpixel ? b.dsub : nullptr;
  a.dbg_sum = b.dbg_sum;
  a.err = b.err;
  a.sc.p1x2 = (uint32_t)k.p1 * 0x10001u;
  a.sc.dpx2 = (uint32_t)(k.p2 - k.p1) * 0x10001u;
  a.lo = b.band_lo;
  a.tw = k.tw;
  a.th = k.th;
  a.gate = b.gate;
  if (k.band) {
    if constexpr (CPL <= 8) {
      if (k.sweep) return launch_rows_v<CPL, S8, 2, true, true>(a, nf, s);
      if (k.num_paths == 8) return launch_rows_v<CPL, S8, 3, true, true>(a, nf, s);
      return launch_rows_v<CPL, S8, 1, true, true>(a, nf, s);
    }
    return cudaErrorInvalidValue;
  }
  const bool fulld = k.D == k.Dp;
  if (k.sweep)
    return fulld ? launch_rows_v<CPL, S8, 2, true, false>(a, nf, s) : launch_rows_v<CPL, S8, 2, false, false>(a, nf, s);
  if (k.num_paths == 8)
    return fulld ? launch_rows_v<CPL, S8, 3, true, false>(a, nf, s) : launch_rows_v<CPL, S8, 3, false, false>(a, nf, s);
  return fulld ? launch_rows_v<CPL, S8, 1, true, false>(a, nf, s) : launch_rows_v<CPL, S8, 1, false, false>(a, nf, s);
}

}  // namespace sgmf

// explicit instantiations of one lane width (CPL cells per lane); the
// instantiating file includes sgmf_sweep.cuh
#define SGMF_AGG_INSTANTIATE(CPL)                                                                        \
  namespace sgmf {                                                                                      \
  template cudaError_t launch_lines_t<CPL, false>(const KParams &, const Buffers &, int, cudaStream_t); \
  template cudaError_t launch_lines_t<CPL, true>(const KParams &, const Buffers &, int, cudaStream_t);  \
  template cudaError_t launch_rows_t<CPL, false>(const KParams &, const Buffers &, int, cudaStream_t);  \
  template cudaError_t launch_rows_t<CPL, true>(const KParams &, const Buffers &, int, cudaStream_t);   \
  template cudaError_t launch_sweep_t<CPL>(const KParams &, const Buffers &, int, cudaStream_t);         \
  template int sweep_plan_t<CPL>(const KParams &, int, int *);                                          \
  }
