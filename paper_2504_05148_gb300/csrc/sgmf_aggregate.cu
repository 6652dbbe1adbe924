// sgmf_aggregate.cu -- SGM path aggregation (Eq. 2), path sum and WTA (Eq. 3).
//
// Lines.  Each of the eight directions of Sec. III runs along a family of
// lines; a line is walked once in each of its two directions by one warp:
//   family 0 (vertical)      line k = column k            down: r=(0,1)   up: r=(0,-1)
//   family 1 (diagonal)      line k: x = (k + y) mod W    down: r=(1,1)   up: r=(-1,-1)
//   family 2 (anti-diagonal) line k: x = (k - y) mod W    down: r=(-1,1)  up: r=(1,-1)
//   rows                     line = row y                 left->right r=(1,0), right->left r=(-1,0)
// With the modulo, every diagonal line has exactly H pixels, and a path
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
// D are padding: their cost is raised to kInf so they never reach the min.
//
// Sums.  The vertical/diagonal kernel writes, per family, the pair sum
// L_down + L_up (u16) of each pixel.  The row kernel adds the two row
// directions and the family sums into S = sum_r L_r and takes d* (Eq. 3)
// and the right-view disparity d' from S on the fly.
#include <cstdint>

#include "sgmf_internal.cuh"

namespace sgmf {

constexpr unsigned kFull = 0xffffffffu;

// ---- lane-vector access ----------------------------------------------------
// u8 cells -> u16x2 words with the pad byte z (0x40 for d >= D) as high byte.
template <int DPL>
struct Vec {
  static constexpr int NW = DPL / 2;
};

template <int DPL>
__device__ __forceinline__ void load_u8(const uint8_t *__restrict__ row, int lane, const uint32_t (&z)[(DPL + 3) / 4],
                                        uint32_t (&w)[DPL / 2]) {
  const uint8_t *p = row + lane * DPL;
  if constexpr (DPL == 2) {
    const uint32_t v = __ldg(reinterpret_cast<const uint16_t *>(p));
    w[0] = prmt(v, z[0], 0x5140);
  } else if constexpr (DPL == 4) {
    const uint32_t v = __ldg(reinterpret_cast<const uint32_t *>(p));
    w[0] = prmt(v, z[0], 0x5140);
    w[1] = prmt(v, z[0], 0x7362);
  } else if constexpr (DPL == 6) {
    const uint16_t *q = reinterpret_cast<const uint16_t *>(p);
    const uint32_t v0 = __ldg(q), v1 = __ldg(q + 1), v2 = __ldg(q + 2);
    // z[0] holds pads of cells 0..3, z[1] of cells 4..5 (bytes 0,1)
    w[0] = prmt(v0, z[0], 0x5140);
    w[1] = prmt(v1, z[0], 0x7160);   // v1.b0, z.b2, v1.b1, z.b3
    w[2] = prmt(v2, z[1], 0x5140);
  } else {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
    w[0] = prmt(v.x, z[0], 0x5140);
    w[1] = prmt(v.x, z[0], 0x7362);
    w[2] = prmt(v.y, z[1], 0x5140);
    w[3] = prmt(v.y, z[1], 0x7362);
  }
}

// u16x2 words -> u8 cells (values known to be <= 255 for real cells)
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
    uint2 v;
    v.x = prmt(w[0], w[1], 0x6420);
    v.y = prmt(w[2], w[3], 0x6420);
    *reinterpret_cast<uint2 *>(p) = v;
  }
}

template <int DPL>
__device__ __forceinline__ void load_u8_plain(const uint8_t *row, int lane, uint32_t (&w)[DPL / 2]) {
  const uint8_t *p = row + lane * DPL;
  if constexpr (DPL == 2) {
    const uint32_t v = *reinterpret_cast<const uint16_t *>(p);
    w[0] = prmt(v, 0, 0x4140);
  } else if constexpr (DPL == 4) {
    const uint32_t v = *reinterpret_cast<const uint32_t *>(p);
    w[0] = prmt(v, 0, 0x4140);
    w[1] = prmt(v, 0, 0x4342);
  } else if constexpr (DPL == 6) {
    const uint16_t *q = reinterpret_cast<const uint16_t *>(p);
    w[0] = prmt(q[0], 0, 0x4140);
    w[1] = prmt(q[1], 0, 0x4140);
    w[2] = prmt(q[2], 0, 0x4140);
  } else {
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    w[0] = prmt(v.x, 0, 0x4140);
    w[1] = prmt(v.x, 0, 0x4342);
    w[2] = prmt(v.y, 0, 0x4140);
    w[3] = prmt(v.y, 0, 0x4342);
  }
}

// u16 cells (one u16x2 word per two cells), offset lane*DPL elements
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

// spill of the first direction's path costs: u8 when every real cost fits
template <int DPL, bool S8>
__device__ __forceinline__ void spill_store(void *base, size_t cell, int lane, const uint32_t (&w)[DPL / 2]) {
  if constexpr (S8)
    store_u8<DPL>(static_cast<uint8_t *>(base) + cell, lane, w);
  else
    store_u16<DPL>(static_cast<uint16_t *>(base) + cell, lane, w);
}

template <int DPL, bool S8>
__device__ __forceinline__ void spill_load(const void *base, size_t cell, int lane, uint32_t (&w)[DPL / 2]) {
  if constexpr (S8)
    load_u8_plain<DPL>(static_cast<const uint8_t *>(base) + cell, lane, w);
  else
    load_u16<DPL>(static_cast<const uint16_t *>(base) + cell, lane, w);
}

// ---- the recursion -----------------------------------------------------------
struct StepConsts {
  uint32_t p1x2;   // P1 in both halves
  uint32_t dpx2;   // (P2 - P1) in both halves
};

// One step of Eq. 2 for the lane's words given m = min_k L(p - r, k).
template <int NW>
__device__ __forceinline__ void sgm_step(uint32_t (&L)[NW], const uint32_t (&C)[NW], uint32_t m,
                                         const StepConsts &sc, int lane) {
  const uint32_t mm = m * 0x10001u;
  const uint32_t cap = mm + sc.dpx2;           // m + P2 - P1 per half
  const uint32_t negmm = 0u - mm;
  uint32_t prev = __shfl_up_sync(kFull, L[NW - 1], 1);
  uint32_t next = __shfl_down_sync(kFull, L[0], 1);
  if (lane == 0) prev = kInf2;
  if (lane == 31) next = kInf2;
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
__device__ __forceinline__ uint32_t warp_min(const uint32_t (&L)[NW]) {
  uint32_t v = L[0];
#pragma unroll
  for (int i = 1; i + 1 < NW; i += 2) v = __vimin3_u16x2(v, L[i], L[i + 1]);
  if constexpr (NW % 2 == 0) v = __vminu2(v, L[NW - 1]);
  const uint32_t s = min(v & 0xffffu, v >> 16);
  return __reduce_min_sync(kFull, s);
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

// ---- vertical and diagonal families -------------------------------------------
struct LineArgs {
  KParams k;
  const uint8_t *cost;
  uint16_t *part[3];
  void *spill;            // [3][W][H][Dp] elements
  StepConsts sc;
};

template <int DPL, bool S8>
__global__ void __launch_bounds__(128) k_agg_lines(const __grid_constant__ LineArgs a) {
  constexpr int NW = DPL / 2;
  const int lane = threadIdx.x & 31;
  const int line = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int fam = blockIdx.y;
  const int W = a.k.W, H = a.k.H, Dp = a.k.Dp;
  if (line >= W) return;
  uint32_t z[(DPL + 3) / 4];
  pad_bytes<DPL>(a.k.D, lane, z);
  const size_t spill_base = ((size_t)fam * W + line) * (size_t)H * Dp;
  auto xof = [&](int y) -> int {
    if (fam == 0) return line;
    int x = fam == 1 ? line + y : line - y;
    x %= W;
    return x < 0 ? x + W : x;
  };
  uint32_t L[NW], C[NW];
  uint32_t m = 0;
  // down: r = (0,1), (1,1), (-1,1)
  for (int y = 0; y < H; ++y) {
    const int x = xof(y);
    load_u8<DPL>(a.cost + ((size_t)y * W + x) * Dp, lane, z, C);
    const bool start = y == 0 || (fam == 1 && x == 0) || (fam == 2 && x == W - 1);
    if (start) {
#pragma unroll
      for (int i = 0; i < NW; ++i) L[i] = C[i];
    } else {
      sgm_step<NW>(L, C, m, a.sc, lane);
    }
    m = warp_min<NW>(L);
    spill_store<DPL, S8>(a.spill, spill_base + (size_t)y * Dp, lane, L);
  }
  // up: r = (0,-1), (-1,-1), (1,-1); emit L_down + L_up
  uint16_t *part = a.part[fam];
  for (int y = H - 1; y >= 0; --y) {
    const int x = xof(y);
    load_u8<DPL>(a.cost + ((size_t)y * W + x) * Dp, lane, z, C);
    const bool start = y == H - 1 || (fam == 1 && x == W - 1) || (fam == 2 && x == 0);
    if (start) {
#pragma unroll
      for (int i = 0; i < NW; ++i) L[i] = C[i];
    } else {
      sgm_step<NW>(L, C, m, a.sc, lane);
    }
    m = warp_min<NW>(L);
    uint32_t Ld[NW];
    spill_load<DPL, S8>(a.spill, spill_base + (size_t)y * Dp, lane, Ld);
#pragma unroll
    for (int i = 0; i < NW; ++i) Ld[i] += L[i];
    store_u16<DPL>(part + ((size_t)y * W + x) * Dp, lane, Ld);
  }
}

// ---- rows, path sum and WTA ----------------------------------------------------
struct RowArgs {
  KParams k;
  const uint8_t *cost;
  const uint16_t *part[3];
  int nparts;
  void *spill;            // [H][W][Dp] elements
  int16_t *dstar, *dprime;
  uint16_t *dbg_sum;
  StepConsts sc;
};

template <int DPL, bool S8>
__global__ void __launch_bounds__(32) k_agg_rows(const __grid_constant__ RowArgs a) {
  constexpr int NW = DPL / 2;
  __shared__ uint32_t ring[256];    // best (S << 8 | d) of right-view pixels x' in flight
  const int lane = threadIdx.x & 31;
  const int y = blockIdx.x;
  const int W = a.k.W, D = a.k.D, Dp = a.k.Dp;
  if (y >= a.k.H) return;
  uint32_t z[(DPL + 3) / 4];
  pad_bytes<DPL>(D, lane, z);
  // per-cell key bytes: b0/b1 = disparities of the word's halves, b2/b3 = 0xff for padding
  uint32_t kb[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const int d0 = lane * DPL + 2 * i;
    kb[i] = (uint32_t)(d0 & 0xff) | ((uint32_t)((d0 + 1) & 0xff) << 8) | (d0 >= D ? 0xff0000u : 0u) |
            (d0 + 1 >= D ? 0xff000000u : 0u);
  }
  const size_t row = (size_t)y * W;
  uint32_t L[NW], C[NW];
  uint32_t m = 0;
  // right -> left: r = (-1, 0)
  for (int x = W - 1; x >= 0; --x) {
    load_u8<DPL>(a.cost + (row + x) * Dp, lane, z, C);
    if (x == W - 1) {
#pragma unroll
      for (int i = 0; i < NW; ++i) L[i] = C[i];
    } else {
      sgm_step<NW>(L, C, m, a.sc, lane);
    }
    m = warp_min<NW>(L);
    spill_store<DPL, S8>(a.spill, (row + x) * Dp, lane, L);
  }
  // left -> right: r = (1, 0), then S, d*, d'
  for (int x = 0; x < W; ++x) {
    const size_t cell = (row + x) * Dp;
    load_u8<DPL>(a.cost + cell, lane, z, C);
    if (x == 0) {
#pragma unroll
      for (int i = 0; i < NW; ++i) L[i] = C[i];
    } else {
      sgm_step<NW>(L, C, m, a.sc, lane);
    }
    m = warp_min<NW>(L);
    uint32_t S[NW], T[NW];
    spill_load<DPL, S8>(a.spill, cell, lane, S);
#pragma unroll
    for (int i = 0; i < NW; ++i) S[i] += L[i];
    for (int j = 0; j < a.nparts; ++j) {
      load_u16<DPL>(a.part[j] + cell, lane, T);
#pragma unroll
      for (int i = 0; i < NW; ++i) S[i] += T[i];
    }
    if (a.dbg_sum != nullptr) store_u16<DPL>(a.dbg_sum + cell, lane, S);
    // keys (S << 8 | d); padding cells get 0xff.. in the top byte
    uint32_t best = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      const uint32_t klo = prmt(S[i], kb[i], 0x6104);
      const uint32_t khi = prmt(S[i], kb[i], 0x7325);
      best = min(best, min(klo, khi));
      // right view: pixel x' = x - d takes S(x, d) as a candidate
      const int d0 = lane * DPL + 2 * i;
      if (d0 < D && x - d0 >= 0) {
        uint32_t *slot = &ring[(x - d0) & 255];
        *slot = d0 == 0 ? klo : min(*slot, klo);
      }
      if (d0 + 1 < D && x - d0 - 1 >= 0) {
        uint32_t *slot = &ring[(x - d0 - 1) & 255];
        *slot = min(*slot, khi);
      }
    }
    best = __reduce_min_sync(kFull, best);
    __syncwarp();
    if (lane == 0) {
      a.dstar[row + x] = (int16_t)(best & 0xffu);
      const int xr = x - (D - 1);
      if (xr >= 0) a.dprime[row + xr] = (int16_t)(ring[xr & 255] & 0xffu);
    }
    __syncwarp();
  }
  // right-view pixels whose diagonal runs off the right border
  for (int xr = max(0, W - D + 1) + lane; xr < W; xr += 32)
    a.dprime[row + xr] = (int16_t)(ring[xr & 255] & 0xffu);
}

template <int DPL, bool S8>
static cudaError_t launch_lines_t(const KParams &k, const Buffers &b, cudaStream_t s) {
  LineArgs a;
  a.k = k;
  a.cost = b.cost;
  for (int i = 0; i < 3; ++i) a.part[i] = b.part[i];
  a.spill = b.spill;
  a.sc.p1x2 = (uint32_t)k.p1 * 0x10001u;
  a.sc.dpx2 = (uint32_t)(k.p2 - k.p1) * 0x10001u;
  dim3 grid((k.W + 3) / 4, k.num_paths == 8 ? 3 : 1);
  k_agg_lines<DPL, S8><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DPL, bool S8>
static cudaError_t launch_rows_t(const KParams &k, const Buffers &b, cudaStream_t s) {
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
  a.sc.p1x2 = (uint32_t)k.p1 * 0x10001u;
  a.sc.dpx2 = (uint32_t)(k.p2 - k.p1) * 0x10001u;
  k_agg_rows<DPL, S8><<<k.H, 32, 0, s>>>(a);
  return cudaGetLastError();
}

#define SGMF_DISPATCH(FN, ...)                                                          \
  switch (k.DPL * 2 + (spill8 ? 1 : 0)) {                                               \
    case 4: return FN<2, false>(__VA_ARGS__);                                           \
    case 5: return FN<2, true>(__VA_ARGS__);                                            \
    case 8: return FN<4, false>(__VA_ARGS__);                                           \
    case 9: return FN<4, true>(__VA_ARGS__);                                            \
    case 12: return FN<6, false>(__VA_ARGS__);                                          \
    case 13: return FN<6, true>(__VA_ARGS__);                                           \
    case 16: return FN<8, false>(__VA_ARGS__);                                          \
    case 17: return FN<8, true>(__VA_ARGS__);                                           \
    default: return cudaErrorInvalidValue;                                              \
  }

cudaError_t launch_agg_lines(const KParams &k, const Buffers &b, bool spill8, cudaStream_t s) {
  SGMF_DISPATCH(launch_lines_t, k, b, s)
}

cudaError_t launch_agg_rows(const KParams &k, const Buffers &b, bool spill8, cudaStream_t s) {
  SGMF_DISPATCH(launch_rows_t, k, b, s)
}

}  // namespace sgmf
