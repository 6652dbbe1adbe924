// sgmf_band.cu -- kernels of the banded mode (not in the paper): the method
// restricted to a disparity band [lo_p, lo_p + B) per pixel, lo_p constant on
// kBandTile x kBandTile pixel tiles.  Ingest, census, semidensification and
// the check are the plain kernels; the cost (here) and the aggregation with
// its WTA (sgmf_aggregate.cuh, BANDED variants) work on the bands.
#include <cstdint>

#include "sgmf_cost.cuh"
#include "sgmf_internal.cuh"

namespace sgmf {

// the caller's band starts, clamped to [0, D - B] so that every band lies in
// [0, D - 1]
__global__ void k_band_clamp(const int16_t *__restrict__ in, int16_t *__restrict__ out, int n, int hi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int16_t)min(max((int)in[i], 0), hi);
}

cudaError_t launch_band_clamp(const KParams &k, const Buffers &b, int nf, const int16_t *lo_in, cudaStream_t s) {
  const int n = nf * k.th * k.tw;
  k_band_clamp<<<(n + 255) / 256, 256, 0, s>>>(lo_in, b.band_lo, n, k.D - k.band);
  return cudaGetLastError();
}

// Banded cost: cell j of pixel p holds C-bar(p, lo_p + j) (Eq. 4, the plain
// rules).  A CTA handles npc pixels of one row (a multiple of the band tile, at
// most kBandCostPx, the row split evenly); the right-census window
// covering all their bands is staged in shared memory VL times, copy kk shifted
// by kk entries, so that a run of entries starting anywhere is a run of whole
// vectors in one copy.  A warp takes four consecutive pixels at a time (they
// lie in one band tile, so they share lo): a lane owns B / 32 consecutive cells
// of each, reads the 3 + B / 32 window entries those need with a few aligned
// vector loads, and stores each pixel's cells as packed bytes straight into the
// banded cost volume (a warp's stores for one pixel are its B contiguous
// bytes).  Pixels with a prior take the far class first; the one or two lanes
// that hold cells with |d - prior| <= 1 then rewrite those.
constexpr int kBandCostPx = 512;

template <typename CT, int B>
__global__ void __launch_bounds__(256) k_cost_banded(KParams k, Buffers b0, const __grid_constant__ CostTable tab,
                                                     int npc) {
  constexpr int DPL = B / 32;
  using CW = CostWin<CT, DPL>;
  constexpr int P = CW::P, VL = CW::VL, NE = CW::NE;
  // a step reads entries up to span + 1 + VL of the window (span below), and
  // span <= npc - 1 + kMaxDisp
  constexpr int NWIN = kBandCostPx + kMaxDisp + 8;
  static_assert(kBandTile % P == 0 && kBandCostPx % kBandTile == 0, "a step's pixels share one band tile");
  static_assert(NWIN * sizeof(CT) % 16 == 0, "every copy starts on a 16-byte boundary");
  __shared__ __align__(16) CT cr_s[VL][NWIN];    // copy kk: cr_s[kk][i] = cR(base + i + kk)
  __shared__ __align__(16) CT cl_s[kBandCostPx];
  __shared__ __align__(16) int16_t pd_s[kBandCostPx];
  __shared__ int lo_s[kBandCostPx / kBandTile];
  __shared__ uint8_t tab_s[4 * 64];
  const Buffers b = frame_view(k, b0, blockIdx.z);
  if (gated_off(b.gate, k.gate_run)) return;
  const int x0 = blockIdx.x * npc, y = blockIdx.y, W = k.W;
  const size_t rowp = (size_t)y * W;
  const CT *cl = static_cast<const CT *>(b.censL) + rowp;
  const CT *cr = static_cast<const CT *>(b.censR) + rowp;
  const int16_t *prior = (k.semidense ? b.dhat : b.dbar) + rowp;
  const int npx = min(npc, W - x0);
  const int ntile = (npx + kBandTile - 1) / kBandTile;
  if (threadIdx.x < npc / kBandTile)
    lo_s[threadIdx.x] =
        threadIdx.x < ntile ? b.band_lo[(y >> kBandTileLog) * k.tw + (x0 >> kBandTileLog) + threadIdx.x] : 0;
  for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x) tab_s[i] = (&tab.v[0][0])[i];
  __syncthreads();
  int lo_min = lo_s[0], lo_max = lo_s[0];
  for (int t = 1; t < ntile; ++t) {
    lo_min = min(lo_min, lo_s[t]);
    lo_max = max(lo_max, lo_s[t]);
  }
  // cR(x - (lo + j)) is entry px + (lo_max - lo) + B - 1 - j of the window
  const int base = x0 - lo_max - (B - 1);
  const int span = (npx - 1) + (lo_max - lo_min) + B;   // entries the cells use
  const int nst = min(span + 8, NWIN);                  // entries staged: all a step reads
#pragma unroll
  for (int kk = 0; kk < VL; ++kk)
    for (int j = threadIdx.x; j < nst; j += blockDim.x) {
      const int xx = base + j + kk;
      cr_s[kk][j] = (xx >= 0 && xx < W) ? cr[xx] : (CT)0;
    }
  for (int i = threadIdx.x; i < npc; i += blockDim.x) {
    const int xx = x0 + i;
    cl_s[i] = xx < W ? cl[xx] : (CT)0;
    pd_s[i] = xx < W ? prior[xx] : (int16_t)-1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int j0 = DPL * lane;                      // the lane's first band cell
  // every pixel of the CTA has x - d >= 0 for all its band cells
  const bool inner = x0 >= lo_max + B - 1;
  uint8_t *out = b.cost + (rowp + x0) * B + j0;
  for (int xb = P * warp; xb < npx; xb += P * nwarp) {
    const int lo = lo_s[xb >> kBandTileLog];
    // cR(x - lo - j) of pixel xb + u and cell j = j0 + i is entry jlo + DPL - 1 + u - i
    const int jlo = xb + (lo_max - lo) + DPL * (31 - lane);
    const int kk = jlo % VL;
    const typename CW::V *run = reinterpret_cast<const typename CW::V *>(&cr_s[kk][jlo - kk]);
    CT e[NE];
#pragma unroll
    for (int q = 0; q < NE / VL; ++q) {
      const typename CW::V t = run[q];
      const CT *tv = reinterpret_cast<const CT *>(&t);
#pragma unroll
      for (int m = 0; m < VL; ++m) e[q * VL + m] = tv[m];
    }
    CT c[P];
    {
      constexpr int CV = 16 / sizeof(CT);
      const uint4 *cv = reinterpret_cast<const uint4 *>(cl_s + xb);
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
      const uint2 t = *reinterpret_cast<const uint2 *>(pd_s + xb);
      pd[0] = (int16_t)(t.x & 0xffffu);
      pd[1] = (int16_t)(t.x >> 16);
      pd[2] = (int16_t)(t.y & 0xffffu);
      pd[3] = (int16_t)(t.y >> 16);
    }
    const int d0 = lo + j0;                       // the lane's first disparity
    uint32_t o[P][DPL];
    if (inner) {
#pragma unroll
      for (int u = 0; u < P; ++u) {
        uint32_t h[DPL];
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
          h[i] = (uint32_t)hamming<CT>(c[u], e[DPL - 1 + u - i]);
          o[u][i] = h[i];
        }
        if (pd[u] >= 0) {
#pragma unroll
          for (int i = 0; i < DPL; ++i) o[u][i] = tab_s[2 * 64 + h[i]];   // far class
          if (pd[u] + 1 >= d0 && pd[u] - 1 < d0 + DPL) {
#pragma unroll
            for (int i = 0; i < DPL; ++i) {
              const int dd = d0 + i - pd[u];
              if (dd >= -1 && dd <= 1) o[u][i] = tab_s[(dd != 0) * 64 + h[i]];
            }
          }
        }
      }
    } else {
      const int x = x0 + xb;
#pragma unroll
      for (int u = 0; u < P; ++u)
#pragma unroll
        for (int i = 0; i < DPL; ++i) {
          const int d = d0 + i;
          const int h = x + u >= d ? hamming<CT>(c[u], e[DPL - 1 + u - i]) : k.nbits;
          const int cls = pd[u] < 0 ? 3 : min(abs(d - pd[u]), 2);
          o[u][i] = tab_s[cls * 64 + h];
        }
    }
#pragma unroll
    for (int u = 0; u < P; ++u)
      if (xb + u < npx) store_cost_bytes<DPL>(out + (size_t)(xb + u) * B, o[u]);
  }
}

template <typename CT>
static void launch_cost_banded_t(const KParams &k, const Buffers &b, int nf, const CostTable &tab, cudaStream_t s) {
  // equal pieces of at most kBandCostPx pixels, rounded up to whole band tiles
  const int n = (k.W + kBandCostPx - 1) / kBandCostPx;
  const int npc = ((k.W + n - 1) / n + kBandTile - 1) / kBandTile * kBandTile;
  dim3 grid((k.W + npc - 1) / npc, k.H, nf);
  if (k.band == 64)
    k_cost_banded<CT, 64><<<grid, 256, 0, s>>>(k, b, tab, npc);
  else
    k_cost_banded<CT, 128><<<grid, 256, 0, s>>>(k, b, tab, npc);
}

cudaError_t launch_cost_banded(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  const CostTable tab = cost_table(k);
  if (k.census == 1)
    launch_cost_banded_t<uint64_t>(k, b, nf, tab, s);
  else
    launch_cost_banded_t<uint32_t>(k, b, nf, tab, s);
  return cudaGetLastError();
}

}  // namespace sgmf
