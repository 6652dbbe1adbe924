// sgmf_band.cu -- kernels of the banded mode (not in the paper): the method
// restricted to a disparity band [lo_p, lo_p + B) per pixel, lo_p constant on
// kBandTile x kBandTile pixel tiles.  Ingest, census, semidensification and the check are
// the plain kernels; the cost, the aggregation (sgmf_aggregate.cuh, BANDED
// variants) and the WTA work on the bands.
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
// rules).  A CTA handles 64 pixels (several tiles) of one row; the right-census
// window covering all their bands is staged in shared memory and the lanes
// of a warp walk the cells of one pixel.
constexpr int kBandCostPx = 64;

template <typename CT, int B>
__global__ void __launch_bounds__(256) k_cost_banded(KParams k, Buffers b0, const __grid_constant__ CostTable tab) {
  __shared__ CT cr_s[kBandCostPx + B + kMaxDisp];
  __shared__ CT cl_s[kBandCostPx];
  __shared__ int pd_s[kBandCostPx];
  __shared__ int lo_s[kBandCostPx / kBandTile];
  __shared__ uint8_t tab_s[4 * 64];
  __shared__ __align__(16) uint8_t out_s[kBandCostPx * B];
  const Buffers b = frame_view(k, b0, blockIdx.z);
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
  // cr_s[i] = cR(base + i) covers x - d for every pixel x and d in its band
  const int base = x0 - lo_max - (B - 1);
  const int span = (npx - 1) + (lo_max - lo_min) + B;   // <= 63 + (D - B) + B
  for (int i = threadIdx.x; i < span; i += blockDim.x) {
    const int xx = base + i;
    cr_s[i] = (xx >= 0 && xx < W) ? cr[xx] : (CT)0;
  }
  if (threadIdx.x < kBandCostPx) {
    const int xx = x0 + threadIdx.x;
    cl_s[threadIdx.x] = xx < W ? cl[xx] : (CT)0;
    pd_s[threadIdx.x] = xx < W ? prior[xx] : -1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int px = warp; px < npx; px += 8) {
    const int x = x0 + px;
    const CT c = cl_s[px];
    const int pd = pd_s[px];
    const int lo = lo_s[px >> kBandTileLog];
#pragma unroll
    for (int m = 0; m < B / 32; ++m) {
      const int j = lane + 32 * m, d = lo + j;
      int h;
      if (x >= d) {
        const CT r = cr_s[x - d - base];
        if constexpr (sizeof(CT) == 4)
          h = __popc(c ^ r);
        else
          h = __popcll(c ^ r);
      } else {
        h = k.nbits;
      }
      const int cls = pd < 0 ? 3 : min(abs(d - pd), 2);
      out_s[px * B + j] = tab_s[cls * 64 + h];
    }
  }
  __syncthreads();
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

// Banded WTA from S: d*_p = lo_p + argmin_j S(p, j) (ties: smaller d), and
// d'(x') = argmin over the cells (x' + d, d) inside the bands (ties: smaller
// d), or -1 where no band holds such a cell.  One CTA per row: a warp takes
// one pixel at a time (lanes over its B cells), keys S << 8 | d; the
// right-view keys are min-merged in shared memory with atomicMin.
template <int B>
__global__ void __launch_bounds__(256) k_wta_banded(KParams k, Buffers b0) {
  extern __shared__ uint32_t keys[];   // [W]
  const Buffers b = frame_view(k, b0, blockIdx.y);
  const int y = blockIdx.x, W = k.W;
  for (int i = threadIdx.x; i < W; i += blockDim.x) keys[i] = 0xffffffffu;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int CL = B / 32;   // cells per lane: 2 or 4
  const int16_t *lo_row = b.band_lo + (size_t)(y >> kBandTileLog) * k.tw;
  for (int x = warp; x < W; x += 8) {
    const int lo = lo_row[x >> kBandTileLog];
    const uint16_t *sp = b.band_sum + ((size_t)y * W + x) * B + lane * CL;
    uint32_t v[CL];
    if constexpr (CL == 2) {
      const uint32_t t = *reinterpret_cast<const uint32_t *>(sp);
      v[0] = t & 0xffffu;
      v[1] = t >> 16;
    } else {
      const uint2 t = *reinterpret_cast<const uint2 *>(sp);
      v[0] = t.x & 0xffffu;
      v[1] = t.x >> 16;
      v[2] = t.y & 0xffffu;
      v[3] = t.y >> 16;
    }
    uint32_t best = 0xffffffffu;
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int d = lo + lane * CL + i;
      const uint32_t key = (v[i] << 8) | (uint32_t)d;
      best = min(best, key);
      if (x - d >= 0) atomicMin(&keys[x - d], key);
    }
    best = __reduce_min_sync(0xffffffffu, best);
    if (lane == 0) b.dstar[(size_t)y * W + x] = (int16_t)(best & 0xffu);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < W; i += blockDim.x)
    b.dprime[(size_t)y * W + i] = keys[i] == 0xffffffffu ? (int16_t)-1 : (int16_t)(keys[i] & 0xffu);
}

cudaError_t launch_wta_banded(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  dim3 grid(k.H, nf);
  const size_t sm = (size_t)k.W * 4;
  if (k.band == 64)
    k_wta_banded<64><<<grid, 256, sm, s>>>(k, b);
  else
    k_wta_banded<128><<<grid, 256, sm, s>>>(k, b);
  return cudaGetLastError();
}

}  // namespace sgmf
