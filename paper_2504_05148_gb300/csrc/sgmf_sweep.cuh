// sgmf_sweep.cuh -- row-synchronous aggregation of the six vertical and
// diagonal directions of Eq. 2 (Sec. III, 8 paths).
//
// The line kernels walk each line of a family separately and read the cost
// volume once per direction.  Here one thread-block cluster sweeps a whole
// frame row by row: the down sweep carries r = (0,1), (1,1), (-1,1) together,
// the up sweep r = (0,-1), (1,-1), (-1,-1), so a sweep reads every cost row
// once for three directions and writes one u16 sum of the three path costs
// per cell (the row kernel adds the two sums and its own two directions).
//
// A row of the frame is split into strips, one per CTA of the cluster, and a
// strip into runs of P pixels, one per 16-lane group.  A group keeps the
// three path-cost vectors of its P pixels in registers.  From one row to the
// next the vertical direction stays on its pixel, the "from-left" diagonal
// (predecessor x - 1) moves one pixel right and the "from-right" diagonal
// (predecessor x + 1) one pixel left, so the only state that crosses a group
// boundary per row is one vector each way.  Those go through shared-memory
// slots, double-buffered by row parity.  Inside a CTA a split row barrier (an
// mbarrier with one arrival per warp) orders them: a group computes the two
// vectors it sends, waits for the previous row's barrier, reads what entered
// it, stores what it sends, arrives, and only then does the rest of the row,
// so the barrier's latency hides behind almost a full row of work.  The
// strip's end groups exchange with the neighbouring CTAs by st.async, whose
// bytes complete on the receiving CTA's message barrier; a pair of groups
// sends its row-t vectors only after receiving the other's row t-1 vectors,
// which is what makes two slots per direction enough.  No thread waits at
// cluster scope inside the row loop.
//
// Cost rows arrive by bulk copies (one per row and CTA: the strip's pixels
// are contiguous) into a ring of R stages, two rows ahead.  Every mbarrier
// wait is bounded (the error word records a timeout); the two cluster
// barriers, at the start and the end, are executed by every thread.
#pragma once

#include <type_traits>

#include "sgmf_aggregate.cuh"

namespace sgmf {

struct SweepArgs {
  KParams k;
  const uint8_t *cost;
  uint16_t *sum[2];       // down / up sweep sums, u16 [F][H][W][Dp]
  int *err;
  StepConsts sc;
  int strip;              // pixels per CTA (= 2 * warps * P)
  const int16_t *lo;      // banded mode: band starts per tile, [frame][th][tw]; null otherwise
  int tw, th;
  const int *gate;        // per-frame gate words of the launch's frames, or null
};

template <int CPL, bool BANDED>
struct SweepCfg {
  static constexpr int Dp = 16 * CPL, NW = CPL / 2;
  // pixels per group and warps per CTA: 8 pixels and 8 warps (202 registers
  // a thread) up to 8 cells per lane -- built for 10 warps it was held to 168
  // registers and ran 8 % slower on the 1242-pixel row; 4 pixels and 20 warps
  // (96 registers) for the banded variant there, whose band bookkeeping would
  // spill at 8; 4 pixels and 10 warps above 8 cells per lane
  static constexpr int P = CPL <= 8 && !BANDED ? 8 : 4;
  static constexpr int kMaxWarps = CPL <= 8 ? (BANDED ? 20 : 8) : 10;
  static constexpr int kMaxCluster = 16;         // CTAs per cluster (above 8: non-portable)
  static constexpr int R = 4;                    // ring stages (rows)
  static constexpr int kSlot = (NW + 1) * 16;    // words of one exchanged vector: NW words + m, per lane
  // at least kExclusive bytes: one CTA per SM, so that the clusters the
  // device holds at once are the SMs the sweep occupies
  static constexpr int kExclusive = 120 * 1024;
  // ring, barriers, exchange slots, one band-shift buffer (Dp u16) and the
  // edge words of its 3P + 2 vectors (two words each) per group
  // the plain sweep's sums leave by bulk copies (Dp <= 128: the buffers fit
  // beside the ring): per warp two staging buffers (by row parity) of its
  // 2 P pixels' u16 sums
  static constexpr bool kBulkSums = !BANDED && CPL <= 8;
  static constexpr int kSumBuf = 2 * P * Dp;   // u16 elements of one buffer
  static constexpr int smem_bytes(int warps) {
    return max(kExclusive, R * (2 * warps * P) * Dp + (R + 5) * 8 + 2 * 2 * (2 * warps) * kSlot * 4 +
                               (2 * warps) * Dp * 2 + (2 * warps) * (3 * P + 2) * 2 * 4 +
                               (kBulkSums ? warps * 2 * kSumBuf * 2 + 128 : 0));
  }
};

// ---- cluster primitives (inline PTX) -----------------------------------------------
// The .aligned forms need the whole warp at the same instruction: each call
// first reconverges the warp.
__device__ __forceinline__ void cluster_arrive() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait() {
  __syncwarp();
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_map(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// asynchronous 4-byte store into (another CTA's) shared memory whose
// completion counts 4 bytes on the mbarrier at mbar (same CTA as addr)
__device__ __forceinline__ void st_async(uint32_t addr, uint32_t v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
               "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int NW>
__device__ __forceinline__ void copy_vec(uint32_t (&dst)[NW], const uint32_t (&src)[NW]) {
#pragma unroll
  for (int w = 0; w < NW; ++w) dst[w] = src[w];
}

// one Eq. 2 step from predecessor (L, m) on costs C: the new vector and its min
template <int NW>
__device__ __forceinline__ void sweep_step(uint32_t (&out)[NW], uint32_t &mout, const uint32_t (&pred)[NW],
                                           uint32_t mpred, const uint32_t (&C)[NW], const StepConsts &sc,
                                           uint32_t edge_lo, uint32_t edge_hi, int grp) {
  copy_vec<NW>(out, pred);
  sgm_step<NW>(out, C, mpred, sc, edge_lo, edge_hi);
  mout = group_min<NW>(out, grp);
}

// the same on the bands, with the predecessor's edge word e (sgm_step_e)
template <int NW>
__device__ __forceinline__ void sweep_step_e(uint32_t (&out)[NW], uint32_t &mout, const uint32_t (&pred)[NW],
                                             uint32_t mpred, const uint32_t (&C)[NW], const StepConsts &sc,
                                             uint32_t e, int lig, int grp) {
  copy_vec<NW>(out, pred);
  sgm_step_e<NW>(out, C, mpred, sc, e, lig);
  mout = group_min<NW>(out, grp);
}

template <int CPL, bool BANDED>
__global__ void __launch_bounds__(32 * SweepCfg<CPL, BANDED>::kMaxWarps, 1)
    k_agg_sweep(const __grid_constant__ SweepArgs a) {
  using CF = SweepCfg<CPL, BANDED>;
  constexpr int P = CF::P, NW = CF::NW, Dp = CF::Dp, R = CF::R, SL = CF::kSlot;
  constexpr uint32_t kMsgBytes = SL * 4;            // one exchanged vector: 16 lanes x (NW + 1) words
  extern __shared__ __align__(128) uint8_t smem[];
  const int W = a.k.W, H = a.k.H, strip = a.strip;
  const int rank = blockIdx.x, ncta = gridDim.x;   // the cluster spans grid.x
  const bool up = blockIdx.y != 0;
  const int f = blockIdx.z;
  // a skipped frame: every CTA of the cluster (one frame) returns before any copy or barrier
  if (gated_off(a.gate ? a.gate + f : nullptr, a.k.gate_run)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 4, lig = lane & 15;
  const int nwarp = blockDim.x >> 5, ng = 2 * nwarp, gi = warp * 2 + grp;
  const int x_cta = rank * strip;
  const int npx = min(strip, W - x_cta);           // >= 1: the cluster has ceil(W / strip) CTAs
  const int xg = x_cta + gi * P;                   // the group's first pixel
  uint8_t *ring = smem;
  // mbarriers: R ring stages, the row barrier of the CTA, and the four
  // message barriers [dir][parity] of the vectors that arrive from the
  // neighbouring CTAs (dir 0: into group 0 from the left, dir 1: into the
  // last group from the right)
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + R * strip * Dp);
  uint64_t *rowbar = bars + R;
  uint64_t *rx = bars + R + 1;
  uint32_t *slots = reinterpret_cast<uint32_t *>(bars + R + 5);   // [dir][parity][group][NW + 1][16]
  uint16_t *shbuf = reinterpret_cast<uint16_t *>(slots + 2 * 2 * ng * SL) + gi * Dp;   // the group's shift scratch
  // banded mode: a group's pixels share one band tile column (groups are 4
  // pixels from a multiple of 4, tiles 8 wide)
  constexpr bool banded = BANDED;
  const int16_t *lo_f = banded ? a.lo + (size_t)f * a.th * a.tw : nullptr;
  auto lo_at = [&](int x, int y) -> int {
    x = min(max(x, 0), W - 1);
    return lo_f[(y >> kBandTileLog) * a.tw + (x >> kBandTileLog)];
  };
  const size_t fcells = frame_cells(a.k);
  const uint8_t *cost = a.cost + f * fcells;
  uint16_t *out = a.sum[up ? 1 : 0] + f * fcells + lig * CPL;

  if (threadIdx.x == 0) {
    for (int s = 0; s < R; ++s) mbar_init(&bars[s], 1);
    mbar_init(rowbar, (uint32_t)nwarp);             // one arrival per warp and row
    for (int i = 0; i < 4; ++i) mbar_init(&rx[i], 1);   // the receiver's expect_tx arrival
    mbar_fence_init();
  }
  __syncthreads();
  int issued = 0;                                  // thread 0: rows whose copy was issued
  auto issue = [&](int t) {
    const int y = up ? H - 1 - t : t;
    mbar_expect_tx(&bars[t % R], (uint32_t)(npx * Dp));
    bulk_g2s(ring + (size_t)(t % R) * strip * Dp, cost + ((size_t)y * W + x_cta) * Dp, (uint32_t)(npx * Dp),
             &bars[t % R]);
    issued = t + 1;
  };
  if (threadIdx.x == 0) {
    issue(0);
    if (H > 1) issue(1);
  }
  // every CTA of the cluster runs, its barriers initialised, before the first remote store
  cluster_arrive();
  cluster_wait();

  uint32_t z[CPL / 4];
  pad_bytes<CPL>(a.k.D, lig, z);
  const uint32_t edge_lo = lig == 0 ? 0xffffffffu : 0u, edge_hi = lig == 15 ? 0xffffffffu : 0u;
  const StepConsts sc = a.sc;
  // path-cost vectors of the group's pixels and their minima: vertical,
  // from-left diagonal (predecessor x - 1), from-right diagonal (x + 1)
  uint32_t V[P][NW], DL[P][NW], DR[P][NW];
  uint32_t mV[P], mL[P], mR[P];
#pragma unroll
  for (int i = 0; i < P; ++i) {
#pragma unroll
    for (int w = 0; w < NW; ++w) V[i][w] = DL[i][w] = DR[i][w] = 0u;
    mV[i] = mL[i] = mR[i] = 0u;
  }
  // where this group's two outgoing vectors go: the neighbouring groups'
  // slots, in this CTA (plain stores) or, for the strip's end groups, in the
  // neighbouring CTA (st.async, completing on that CTA's message barrier)
  auto slot = [&](int dir, int par, int g) { return slots + ((dir * 2 + par) * ng + g) * SL + lig; };
  const bool remote_r = gi == ng - 1, remote_l = gi == 0;
  const bool send_r = !remote_r || rank + 1 < ncta, send_l = !remote_l || rank > 0;
  const uint32_t rk_r = remote_r && send_r ? rank + 1 : rank, rk_l = remote_l && send_l ? rank - 1 : rank;
  const int g_r = remote_r ? 0 : gi + 1, g_l = remote_l ? ng - 1 : gi - 1;
  const uint32_t dst_r0 = cluster_map(smem_u32(slot(0, 0, g_r)), rk_r);
  const uint32_t dst_r1 = cluster_map(smem_u32(slot(0, 1, g_r)), rk_r);
  const uint32_t dst_l0 = cluster_map(smem_u32(slot(1, 0, g_l)), rk_l);
  const uint32_t dst_l1 = cluster_map(smem_u32(slot(1, 1, g_l)), rk_l);
  const uint32_t mb_r0 = cluster_map(smem_u32(&rx[0]), rk_r), mb_r1 = cluster_map(smem_u32(&rx[1]), rk_r);
  const uint32_t mb_l0 = cluster_map(smem_u32(&rx[2]), rk_l), mb_l1 = cluster_map(smem_u32(&rx[3]), rk_l);
  // vectors that arrive from another CTA: group 0 from the left, the last group from the right
  const bool recv_l = gi == 0 && rank > 0, recv_r = gi == ng - 1 && rank + 1 < ncta;
  // path starts at the image border: pixel 0's left predecessor is x = -1
  // at the strip of x = 0; a pixel's right predecessor x + 1 = W does not exist
  const uint32_t keep_in_l = xg == 0 ? 0u : 0xffffffffu;
  // warps whose groups touch neither border need none of the masks below
  const bool plain = __all_sync(kFull, xg > 0 && xg + P < W);
  // one Eq. 2 step from a predecessor vector; on the bands with the
  // predecessor's edge word (all ones but on the first step after a shift)
  auto step = [&](uint32_t(&o)[NW], uint32_t &mo, const uint32_t(&pr)[NW], uint32_t mp, const uint32_t(&Cc)[NW],
                  uint32_t e) {
    if constexpr (BANDED)
      sweep_step_e<NW>(o, mo, pr, mp, Cc, sc, e, lig, grp);
    else
      sweep_step<NW>(o, mo, pr, mp, Cc, sc, edge_lo, edge_hi, grp);
  };
  bool ok = true;
  auto bounded = [&](uint64_t *bar, uint32_t parity) {
    if (!mbar_wait_bounded(bar, parity, kWaitLimit)) {
      set_error(a.err, kErrTimeout);
      ok = false;
    }
  };

  // banded: the edge words of the group's vectors on a row that re-indexes
  // them (sgm_step_e), [vector][lane 0 / lane 15]: V[i] = i, DL[i] = P + i,
  // DR[i] = 2P + i, the vector entering from the left 3P, from the right 3P + 1
  constexpr int NE = 3 * P + 2;
  uint32_t *esm0 = reinterpret_cast<uint32_t *>(reinterpret_cast<uint16_t *>(slots + 2 * 2 * ng * SL) + ng * Dp);
  uint32_t *esm = esm0 + gi * NE * 2 + (lig == 15 ? 1 : 0);
  // the warp's sum staging buffers (kBulkSums), after the edge words, 128-byte aligned
  uint16_t *wsum = reinterpret_cast<uint16_t *>((reinterpret_cast<uintptr_t>(esm0 + ng * NE * 2) + 127) &
                                                ~uintptr_t(127)) +
                   (size_t)warp * 2 * CF::kSumBuf;
  uint16_t *sum_base = a.sum[up ? 1 : 0] + f * fcells;   // the launch frame's sums
  const int xw = x_cta + warp * 2 * P;                   // the warp's first pixel
  const int nvw = max(0, min(2 * P, W - xw));            // its pixels inside the image
  // re-index a vector to this row's band and record its edge word (lanes 0 and 15)
  auto shift_rec = [&](uint32_t(&v)[NW], int delta, int k) {
    uint32_t e = 0xffffffffu;
    band_shift<CPL>(v, delta, shbuf, lig, e);
    if (lig == 0 || lig == 15) esm[2 * k] = e;
  };

  for (int t = 0; t < H; ++t) {
    bounded(&bars[t % R], (uint32_t)(t / R) & 1u);
    const uint8_t *st = ring + (size_t)(t % R) * strip * Dp + gi * P * Dp + lig * CPL;
    const int y = up ? H - 1 - t : t, yp = up ? y + 1 : y - 1;   // this row, the previous one
    int delta = 0, dl = 0, dr = 0;
    bool shifted = false;
    if constexpr (BANDED) {
      // the band change of the group's own vectors (a new band tile row) and
      // of the vectors entering from the neighbours (pixel x - 1 or x + P of
      // the previous row, in their own bands)
      const int lo_cur = lo_at(xg, y);
      if (t > 0) {
        delta = lo_cur - lo_at(xg, yp);
        dl = lo_cur - lo_at(xg - 1, yp);
        dr = lo_cur - lo_at(xg + P, yp);
      }
      shifted = __any_sync(kFull, delta != 0 || dl != 0 || dr != 0);
      if (shifted) {
        if (lig == 0 || lig == 15) {
#pragma unroll
          for (int k = 0; k < NE; ++k) esm[2 * k] = 0xffffffffu;
        }
        // every vector of the group moves to the new band (cells without a
        // counterpart in the old band become absent; the old cell just
        // outside the new band goes to the edge word)
        if (__any_sync(kFull, delta != 0)) {
#pragma unroll
          for (int i = 0; i < P; ++i) {
            shift_rec(V[i], delta, i);
            shift_rec(DL[i], delta, P + i);
            shift_rec(DR[i], delta, 2 * P + i);
          }
        }
      }
    }
    // the row's work; E: with the edge words of a re-indexing row
    auto row = [&](auto edges) {
      constexpr bool E = decltype(edges)::value;
      auto edge = [&](int k) -> uint32_t {
        if constexpr (E)
          return esm[2 * k];
        else
          return 0xffffffffu;
      };
      uint32_t C0[NW], CP[NW];
      unpack_u8<CPL>(st, z, C0);
      unpack_u8<CPL>(st + (P - 1) * Dp, z, CP);
      // the two vectors this group sends: from-left of its last pixel (from
      // its own pixel P-2), from-right of its first pixel (from its pixel 1)
      uint32_t eL[NW], eR[NW], meL, meR;
      {
        uint32_t pr[NW], mpr = mR[1];
        copy_vec<NW>(pr, DR[1]);
        if (!plain) {
          const uint32_t kr = xg + 1 < W ? 0xffffffffu : 0u;   // pixel 0's right predecessor inside
#pragma unroll
          for (int w = 0; w < NW; ++w) pr[w] &= kr;
          mpr &= kr;
        }
        step(eL, meL, DL[P - 2], mL[P - 2], CP, edge(2 * P - 2));
        step(eR, meR, pr, mpr, C0, edge(2 * P + 1));
      }
      // the vectors entering this group from the previous row
      uint32_t inL[NW], inR[NW], minL = 0u, minR = 0u;
#pragma unroll
      for (int w = 0; w < NW; ++w) inL[w] = inR[w] = 0u;
      if (t > 0) {
        const int par = (t - 1) & 1;
        // every warp of the CTA has stored row t - 1's vectors (and finished row t - 2)
        bounded(rowbar, (uint32_t)(t - 1) & 1u);
        if (recv_l || recv_r) {
          uint64_t *mb = &rx[(recv_l ? 0 : 1) * 2 + par];
          if (lig == 0) mbar_expect_tx(mb, kMsgBytes);
          bounded(mb, (uint32_t)((t - 1) >> 1) & 1u);
        }
        const uint32_t *sl = slot(0, par, gi), *sr = slot(1, par, gi);
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          inL[w] = sl[w * 16];
          inR[w] = sr[w * 16];
        }
        minL = sl[NW * 16];
        minR = sr[NW * 16];
        if constexpr (E) {
          if (__any_sync(kFull, dl != 0)) shift_rec(inL, dl, 3 * P);
          if (__any_sync(kFull, dr != 0)) shift_rec(inR, dr, 3 * P + 1);
        }
      }
      // the ring stage of row t - 2 is free: every warp finished that row before its row t - 1 arrival
      if (threadIdx.x == 0 && issued < H && issued <= t + 2) issue(issued);
      if (t + 1 < H) {
        // row t's outgoing vectors (the last row's have no reader)
        const int par = t & 1;
        if (send_r) {
          if (remote_r) {
            const uint32_t dst = par ? dst_r1 : dst_r0, mb = par ? mb_r1 : mb_r0;
#pragma unroll
            for (int w = 0; w < NW; ++w) st_async(dst + w * 64, eL[w], mb);
            st_async(dst + NW * 64, meL, mb);
          } else {
            uint32_t *d = slot(0, par, g_r);
#pragma unroll
            for (int w = 0; w < NW; ++w) d[w * 16] = eL[w];
            d[NW * 16] = meL;
          }
        }
        if (send_l) {
          if (remote_l) {
            const uint32_t dst = par ? dst_l1 : dst_l0, mb = par ? mb_l1 : mb_l0;
#pragma unroll
            for (int w = 0; w < NW; ++w) st_async(dst + w * 64, eR[w], mb);
            st_async(dst + NW * 64, meR, mb);
          } else {
            uint32_t *d = slot(1, par, g_l);
#pragma unroll
            for (int w = 0; w < NW; ++w) d[w * 16] = eR[w];
            d[NW * 16] = meR;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(rowbar);
      // the rest of the row
      if (!plain) {
        const uint32_t kl = keep_in_l, kr = xg + P < W ? 0xffffffffu : 0u;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          inL[w] &= kl;
          inR[w] &= kr;
        }
        minL &= kl;
        minR &= kr;
      }
      uint32_t carry[NW], mcarry = mL[0];
      copy_vec<NW>(carry, DL[0]);
      step(DL[0], mL[0], inL, minL, C0, edge(3 * P));
#pragma unroll
      for (int i = 0; i < P; ++i) {
        uint32_t C[NW];
        if (i == 0)
          copy_vec<NW>(C, C0);
        else if (i == P - 1)
          copy_vec<NW>(C, CP);
        else
          unpack_u8<CPL>(st + i * Dp, z, C);
        uint32_t mtmp;
        step(V[i], mtmp, V[i], mV[i], C, edge(i));
        mV[i] = mtmp;
        if (i >= 1 && i <= P - 2) {
          uint32_t nxt[NW];
          const uint32_t mnxt = mL[i];
          copy_vec<NW>(nxt, DL[i]);
          step(DL[i], mL[i], carry, mcarry, C, edge(P + i - 1));
          copy_vec<NW>(carry, nxt);
          mcarry = mnxt;
          uint32_t pr[NW], mpr = mR[i + 1];
          copy_vec<NW>(pr, DR[i + 1]);
          if (!plain) {
            const uint32_t ki = xg + i + 1 < W ? 0xffffffffu : 0u;
#pragma unroll
            for (int w = 0; w < NW; ++w) pr[w] &= ki;
            mpr &= ki;
          }
          step(DR[i], mR[i], pr, mpr, C, edge(2 * P + i + 1));
        } else if (i == 0) {
          copy_vec<NW>(DR[0], eR);
          mR[0] = meR;
        } else {
          copy_vec<NW>(DL[P - 1], eL);
          mL[P - 1] = meL;
          step(DR[P - 1], mR[P - 1], inR, minR, C, edge(3 * P + 1));
        }
        const int x = xg + i;
        if constexpr (CF::kBulkSums) {
          // into the row's staging buffer (pixels outside the image are not copied out)
          uint32_t sum[NW];
#pragma unroll
          for (int w = 0; w < NW; ++w) sum[w] = V[i][w] + DL[i][w] + DR[i][w];
          store_u16<CPL>(wsum + (t & 1) * CF::kSumBuf + (grp * P + i) * Dp + lig * CPL, sum);
        } else if (ok && x < W) {
          uint32_t sum[NW];
#pragma unroll
          for (int w = 0; w < NW; ++w) sum[w] = V[i][w] + DL[i][w] + DR[i][w];
          store_u16<CPL>(out + ((size_t)y * W + x) * Dp, sum);
        }
      }
    };
    if (BANDED && shifted)
      row(std::true_type{});
    else
      row(std::false_type{});
    if constexpr (CF::kBulkSums) {
      // the row's sums of the warp's pixels: one bulk copy from the staging
      // buffer; the buffer of row t - 1 has been read before row t + 1 reuses it
      fence_proxy_async_shared();
      __syncwarp();
      if (lane == 0) {
        if (ok && nvw > 0)
          bulk_s2g(sum_base + ((size_t)y * W + xw) * Dp, wsum + (t & 1) * CF::kSumBuf, (uint32_t)(nvw * Dp * 2));
        bulk_commit();
        bulk_wait_read_all_but_one();
      }
      __syncwarp();
    }
  }
  if constexpr (CF::kBulkSums) {
    if (lane == 0) bulk_wait_all();
  }
  // every message was waited for by its receiver; the cluster barrier keeps
  // every CTA (and its shared memory) alive until all are done
  cluster_arrive();
  cluster_wait();
  if (threadIdx.x == 0 && !ok) {
    for (int h = max(0, issued - R); h < issued; ++h)
      mbar_wait_bounded(&bars[h % R], (uint32_t)(h / R) & 1u, kWaitLimit);
  }
}

// Warps per CTA when a row of W pixels is split over `ctas` CTAs, or 0 when
// that split is not allowed (a CTA above kMaxWarps, or an empty last CTA).
template <int CPL, bool BANDED>
inline int sweep_warps(int W, int ctas) {
  using CF = SweepCfg<CPL, BANDED>;
  if (ctas < 1 || ctas > CF::kMaxCluster) return 0;
  const int warps = (W + ctas * 2 * CF::P - 1) / (ctas * 2 * CF::P);
  if (warps > CF::kMaxWarps || (ctas - 1) * 2 * warps * CF::P >= W) return 0;
  return warps;
}

template <int CPL, bool BANDED>
static cudaLaunchConfig_t sweep_config(int nf, int ctas, int warps, cudaStream_t s, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas, 2, nf);
  cfg.blockDim = dim3(32 * warps);
  cfg.dynamicSmemBytes = SweepCfg<CPL, BANDED>::smem_bytes(warps);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = ctas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// kernel attributes (once per device): the dynamic shared memory and cluster
// sizes above the portable 8
template <int CPL, bool BANDED>
static cudaError_t sweep_attributes() {
  static bool done[64] = {};
  return once_per_device(done, [](int) {
    cudaError_t e = cudaFuncSetAttribute(k_agg_sweep<CPL, BANDED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SweepCfg<CPL, BANDED>::smem_bytes(SweepCfg<CPL, BANDED>::kMaxWarps));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_agg_sweep<CPL, BANDED>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
  });
}

// The cluster size (CTAs per cluster) for the sweep of a context that runs
// up to nb frames per call, or 0 when it cannot run (8 paths only).  A call is 2 nb cluster jobs of H rows each; with n
// clusters resident at once it takes ceil(2 nb / n) waves, and a row takes
// time in proportion to the pixels of one CTA (one CTA per SM).  Among the
// sizes from the smallest that holds a row up to twice that (at most 16) the
// one with the fewest waves x pixels per CTA (ties: the smaller cluster).
template <int CPL, bool BANDED>
static int sweep_plan_b(const KParams &k, int nb, int *slots) {
  using CF = SweepCfg<CPL, BANDED>;
  if (k.num_paths != 8) return 0;
  const int lo = (k.W + 2 * CF::kMaxWarps * CF::P - 1) / (2 * CF::kMaxWarps * CF::P);
  if (lo > CF::kMaxCluster || sweep_attributes<CPL, BANDED>() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int best = 0, best_n = 0;
  long best_cost = 0;
  for (int cs = lo; cs <= min(CF::kMaxCluster, 2 * lo); ++cs) {
    const int warps = sweep_warps<CPL, BANDED>(k.W, cs);
    if (warps == 0) continue;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = sweep_config<CPL, BANDED>(1, cs, warps, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_agg_sweep<CPL, BANDED>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (n < 1) continue;
    const long cost = (long)((2 * nb + n - 1) / n) * (2 * warps * CF::P);
    if (best == 0 || cost < best_cost) {
      best_cost = cost;
      best = cs;
      best_n = n;
    }
  }
  if (slots != nullptr) *slots = best_n;
  return best;
}

template <int CPL>
int sweep_plan_t(const KParams &k, int nb, int *slots) {
  return k.band ? sweep_plan_b<CPL, true>(k, nb, slots) : sweep_plan_b<CPL, false>(k, nb, slots);
}

template <int CPL, bool BANDED>
static cudaError_t launch_sweep_b(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  using CF = SweepCfg<CPL, BANDED>;
  const int ctas = k.sweep_cs, warps = sweep_warps<CPL, BANDED>(k.W, ctas);
  if (warps == 0) return cudaErrorInvalidValue;
  cudaError_t e = sweep_attributes<CPL, BANDED>();
  if (e != cudaSuccess) return e;
  SweepArgs a;
  a.k = lane_params(k);                  // banded: lane cells are band positions
  a.cost = b.cost;
  a.lo = BANDED ? b.band_lo : nullptr;
  a.tw = k.tw;
  a.th = k.th;
  a.sum[0] = b.part[0];
  a.sum[1] = b.part[1];
  a.err = b.err;
  a.gate = b.gate;
  a.sc.p1x2 = (uint32_t)k.p1 * 0x10001u;
  a.sc.dpx2 = (uint32_t)(k.p2 - k.p1) * 0x10001u;
  a.strip = 2 * warps * CF::P;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = sweep_config<CPL, BANDED>(nf, ctas, warps, s, attr);
  return cudaLaunchKernelEx(&cfg, k_agg_sweep<CPL, BANDED>, a);
}

template <int CPL>
cudaError_t launch_sweep_t(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  return k.band ? launch_sweep_b<CPL, true>(k, b, nf, s) : launch_sweep_b<CPL, false>(k, b, nf, s);
}

}  // namespace sgmf
