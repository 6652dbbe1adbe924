// sgmf_cost.cuh -- the joint cost C-bar of Eq. 4 for four consecutive pixels
// of one row, one lane's DPL disparities, from staged census words (the
// step of the cost kernel, which stores the bytes in the cost volume).
//
// H(p,d) = popcount(cL(x,y) ^ cR(x-d,y)), or the number of census bits where
// x - d < 0.  Where the prior (d-hat, or d-bar for DSGM) is invalid C-bar = H;
// otherwise
//   C-bar = floor(((b-a) H + a q + floor(b/2)) / b),  q = 0 / q1 / q2 for
// |d - prior| = 0 / 1 / > 1, looked up in the table (class 2 = far, 3 = none).
// Cells d >= D hold 0.
#pragma once

#include <cstdint>
#include <type_traits>

#include "sgmf_internal.cuh"

namespace sgmf {

constexpr int kCostPix = 4;   // pixels a lane takes at a time

template <typename CT, int DPL>
struct CostWin {
  static constexpr int P = kCostPix;
  static constexpr int VL = sizeof(CT) == 8 ? 2 : (DPL % 4 == 0 ? 4 : 2);   // entries per vector load
  using V = typename std::conditional<VL * sizeof(CT) == 16, uint4, uint2>::type;
  static constexpr int NE = (P + DPL - 1 + VL - 1) / VL * VL;             // entries loaded (= P + DPL)
  static_assert(P % 4 == 0 && DPL % 2 == 0, "aligned window, census and prior loads");
};

// Staged pixels xb .. xb + 3 (xb a multiple of 4; x the first one's image
// column) for the lane's disparities d0 = DPL * lane .. d0 + DPL - 1:
//   cr[j] = cR(xs - (32 DPL - 1) + j), xs the image column of staged pixel 0
//   cl[i] = cL of staged pixel i, pd[i] its prior (-1: none), both 16-byte
//   aligned with cl 16 and pd 8 bytes per four pixels;
// tab: the cost table [4][64] in shared memory.  o[u][i] = C-bar(x + u, d0 + i).
// The P + DPL - 1 entries cR(x + u - d) of the lane are consecutive and start
// on a vector boundary (x - d0 is a multiple of 4 from the window's start),
// so they come from a few aligned vector loads indexed with constants.
template <typename CT, int DPL>
__device__ __forceinline__ void cost_quad(const CT *cr, const CT *cl, const int16_t *pd_s, int xb, int x, int lane,
                                          int D, int nbits, const uint8_t *tab, uint32_t (&o)[kCostPix][DPL]) {
  using CW = CostWin<CT, DPL>;
  constexpr int Dp = 32 * DPL, P = CW::P, VL = CW::VL, NE = CW::NE;
  const int d0 = DPL * lane;
  // cR(x - d) for pixel xb + u and d = d0 + i is entry jlo + DPL - 1 + u - i
  const int jlo = xb + DPL * (31 - lane);
  CT e[NE];
#pragma unroll
  for (int q = 0; q < NE / VL; ++q) {
    const typename CW::V t = reinterpret_cast<const typename CW::V *>(cr + jlo)[q];
    const CT *tv = reinterpret_cast<const CT *>(&t);
#pragma unroll
    for (int m = 0; m < VL; ++m) e[q * VL + m] = tv[m];
  }
  CT c[P];
  {
    constexpr int CV = 16 / sizeof(CT);
    const uint4 *cv = reinterpret_cast<const uint4 *>(cl + xb);
#pragma unroll
    for (int q = 0; q < P / CV; ++q) {
      const uint4 t = cv[q];
      const CT *tv = reinterpret_cast<const CT *>(&t);
#pragma unroll
      for (int m = 0; m < CV; ++m) c[q * CV + m] = tv[m];
    }
  }
  int pd[P];
  {
    const uint2 *pv = reinterpret_cast<const uint2 *>(pd_s + xb);
#pragma unroll
    for (int q = 0; q < P / 4; ++q) {
      const uint2 t = pv[q];
      pd[4 * q] = (int16_t)(t.x & 0xffffu);
      pd[4 * q + 1] = (int16_t)(t.x >> 16);
      pd[4 * q + 2] = (int16_t)(t.y & 0xffffu);
      pd[4 * q + 3] = (int16_t)(t.y >> 16);
    }
  }
  if (D == Dp) {
    // every d is a real disparity; near the left border (x < Dp - 1, the
    // first pixels of a row only) the cells with x - d < 0 take the full
    // census length: a separate copy of the step, so that the others carry no
    // per-cell select
    auto quad = [&](auto border) {
      constexpr bool EDGE = decltype(border)::value;
#pragma unroll
      for (int u = 0; u < P; ++u) {
        uint32_t h[DPL];
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
          h[i] = (uint32_t)hamming<CT>(c[u], e[DPL - 1 + u - i]);
          if (EDGE && x + u < d0 + i) h[i] = (uint32_t)nbits;
          o[u][i] = h[i];
        }
        if (pd[u] >= 0) {
          // the far class for every cell, then the (at most three) cells with
          // |d - prior| <= 1, in the one or two lanes that hold them
#pragma unroll
          for (int i = 0; i < DPL; ++i) o[u][i] = tab[2 * 64 + h[i]];
          if (pd[u] + 1 >= d0 && pd[u] - 1 < d0 + DPL) {
#pragma unroll
            for (int i = 0; i < DPL; ++i) {
              const int dd = d0 + i - pd[u];
              if (dd >= -1 && dd <= 1) o[u][i] = tab[(dd != 0) * 64 + h[i]];
            }
          }
        }
      }
    };
    if (x < Dp - 1)
      quad(std::true_type{});
    else
      quad(std::false_type{});
  } else {
#pragma unroll
    for (int u = 0; u < P; ++u)
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        const int d = d0 + i;
        const int h = x + u >= d ? hamming<CT>(c[u], e[DPL - 1 + u - i]) : nbits;
        const int cls = pd[u] < 0 ? 3 : min(abs(d - pd[u]), 2);
        o[u][i] = d < D ? tab[cls * 64 + h] : 0u;
      }
  }
}

}  // namespace sgmf
