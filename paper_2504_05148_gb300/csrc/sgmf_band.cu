// sgmf_band.cu -- kernels of the banded mode (not in the paper): the method
// restricted to a disparity band [lo_p, lo_p + B) per pixel, lo_p constant on
// kBandTile x kBandTile pixel tiles.  Ingest, census, semidensification and
// the check are the plain kernels; the cost (here) and the aggregation with
// its WTA (sgmf_aggregate.cuh, BANDED variants) work on the bands.
#include <cstdint>

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
// rules).  A CTA handles 128 pixels (several tiles) of one row; the right-census
// window covering all their bands is staged in shared memory, VL times with
// shifts as in the plain cost kernel, and a lane of a warp owns B / 32
// consecutive cells of one pixel, read as one aligned vector and stored as
// packed bytes.  Pixels with a prior take the far class in the loop; one
// thread per pixel rewrites the (at most three) cells with |d - prior| <= 1.
constexpr int kBandCostPx = 128;

template <typename CT, int B>
__global__ void __launch_bounds__(256) k_cost_banded(KParams k, Buffers b0, const __grid_constant__ CostTable tab) {
  constexpr int DPL = B / 32;
  using CV = CostVec<CT, DPL>;
  constexpr int VL = CV::VL, NV = DPL / VL;
  constexpr int NWIN = kBandCostPx + kMaxDisp;    // >= the window span, kBandCostPx - 1 + D
  __shared__ __align__(16) CT cr_s[VL][NWIN];    // copy k: cr_s[k][i] = cR(base + i + k)
  __shared__ CT cl_s[kBandCostPx];
  __shared__ int pd_s[kBandCostPx];
  __shared__ int lo_s[kBandCostPx / kBandTile];
  __shared__ uint8_t tab_s[4 * 64];
  __shared__ __align__(16) uint8_t out_s[kBandCostPx * B];
  const Buffers b = frame_view(k, b0, blockIdx.z);
  if (gated_off(b.gate, k.gate_run)) return;
  const int x0 = blockIdx.x * kBandCostPx, y = blockIdx.y, W = k.W;
  const size_t rowp = (size_t)y * W;
  const CT *cl = static_cast<const CT *>(b.censL) + rowp;
  const CT *cr = static_cast<const CT *>(b.censR) + rowp;
  const int16_t *prior = (k.semidense ? b.dhat : b.dbar) + rowp;
  const int npx = min(kBandCostPx, W - x0);
  const int ntile = (npx + kBandTile - 1) / kBandTile;
  if (threadIdx.x < kBandCostPx / kBandTile)
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
  const int span = (npx - 1) + (lo_max - lo_min) + B;   // <= kBandCostPx - 1 + D
#pragma unroll
  for (int kk = 0; kk < VL; ++kk)
    for (int j = threadIdx.x; j < span - kk; j += blockDim.x) {
      const int xx = base + j + kk;
      cr_s[kk][j] = (xx >= 0 && xx < W) ? cr[xx] : (CT)0;
    }
  if (threadIdx.x < kBandCostPx) {
    const int xx = x0 + threadIdx.x;
    cl_s[threadIdx.x] = xx < W ? cl[xx] : (CT)0;
    pd_s[threadIdx.x] = xx < W ? prior[xx] : -1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = DPL * lane;                      // the lane's first cell
  // every pixel of the CTA has x - d >= 0 for all its band cells
  const bool inner = x0 >= lo_max + B - 1;
  for (int px = warp; px < npx; px += 8) {
    const int x = x0 + px;
    const CT c = cl_s[px];
    const int pd = pd_s[px];
    const int lo = lo_s[px >> kBandTileLog];
    // the lane's run: entries of cells c0 + DPL - 1 .. c0, on a vector boundary of copy kk
    const int off = px + lo_max - lo;
    const int kk = off % VL;
    const CT *run = &cr_s[kk][off + B - DPL * (lane + 1) - kk];
    CT v[DPL];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const typename CV::V t = reinterpret_cast<const typename CV::V *>(run)[q];
      const CT *e = reinterpret_cast<const CT *>(&t);
#pragma unroll
      for (int m = 0; m < VL; ++m) v[q * VL + m] = e[m];
    }
    uint32_t out[DPL];
    if (inner) {
#pragma unroll
      for (int i = 0; i < DPL; ++i) out[i] = (uint32_t)hamming<CT>(c, v[DPL - 1 - i]);
      if (pd >= 0) {
#pragma unroll
        for (int i = 0; i < DPL; ++i) out[i] = tab_s[2 * 64 + out[i]];   // far class; near cells below
      }
    } else {
#pragma unroll
      for (int i = 0; i < DPL; ++i) {
        const int d = lo + c0 + i;
        const int h = x >= d ? hamming<CT>(c, v[DPL - 1 - i]) : k.nbits;
        const int cls = pd < 0 ? 3 : min(abs(d - pd), 2);
        out[i] = tab_s[cls * 64 + h];
      }
    }
    store_cost_bytes<DPL>(out_s + px * B + c0, out);
  }
  __syncthreads();
  if (inner && threadIdx.x < npx) {
    const int px = threadIdx.x, pd = pd_s[px], lo = lo_s[px >> kBandTileLog];
    if (pd >= 0) {
      const CT c = cl_s[px];
#pragma unroll
      for (int j = -1; j <= 1; ++j) {
        const int cell = pd + j - lo;
        if (cell >= 0 && cell < B)
          out_s[px * B + cell] = tab_s[abs(j) * 64 + hamming<CT>(c, cr_s[0][px + lo_max - lo + B - 1 - cell])];
      }
    }
  }
  __syncthreads();
  // the block's [npx][B] bytes are contiguous in the banded cost volume
  uint4 *dst = reinterpret_cast<uint4 *>(b.cost + (rowp + x0) * B);
  const uint4 *src = reinterpret_cast<const uint4 *>(out_s);
  for (int i = threadIdx.x; i < npx * B / 16; i += blockDim.x) dst[i] = src[i];
}

template <typename CT>
static void launch_cost_banded_t(const KParams &k, const Buffers &b, int nf, const CostTable &tab, cudaStream_t s) {
  dim3 grid((k.W + kBandCostPx - 1) / kBandCostPx, k.H, nf);
  if (k.band == 64)
    k_cost_banded<CT, 64><<<grid, 256, 0, s>>>(k, b, tab);
  else
    k_cost_banded<CT, 128><<<grid, 256, 0, s>>>(k, b, tab);
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
