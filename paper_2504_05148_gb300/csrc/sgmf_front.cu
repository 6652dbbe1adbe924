// sgmf_front.cu -- the stages before aggregation (sm_103a):
//   k_ingest      sparse LiDAR map d-bar + presence masks + pitched image copies
//   k_census      9x7 census of both images, windows staged in shared memory by TMA
//   k_boxor_*     separable OR of presence masks over a (2r+1)^2 window
//   k_semidense   Eq. 5
//   k_cost        Hamming cost + DDC, Eq. 4, materialised as uint8 [H][W][Dp]
#include <cuda.h>
#include <cstdint>

#include "sgmf_internal.cuh"

namespace sgmf {

// --------------------------------------------------------------------------
// d-bar (Sec. IV: integer sparse disparity aligned with the left view).
// A LiDAR value f becomes rint(f) (round half to even) when f is finite,
// f > 0 and rint(f) <= D-1; everything else is invalid (-1).  The presence
// mask of a pixel has bit d-bar set.  The images are copied into pitched
// buffers whose rows start on 16-byte boundaries, as TMA requires.
__global__ void __launch_bounds__(256) k_ingest(KParams k, Buffers b0, const uint8_t *__restrict__ left,
                                                const uint8_t *__restrict__ right,
                                                const float *__restrict__ lidar) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= k.W || y >= k.H) return;
  const int f = blockIdx.z;
  const Buffers b = frame_view(k, b0, f);
  const size_t fo = (size_t)f * frame_px(k);
  left += fo;
  right += fo;
  if (lidar != nullptr) lidar += fo;
  const size_t p = (size_t)y * k.W + x;
  int v = -1;
  if (lidar != nullptr) {
    const float f = lidar[p];
    if (isfinite(f) && f > 0.0f) {
      const float r = rintf(f);
      if (r <= (float)(k.D - 1)) v = (int)r;
    }
  }
  b.dbar[p] = (int16_t)v;
  const size_t plane = (size_t)k.W * k.H;
  for (int w = 0; w < k.MW; ++w)
    b.pres[w * plane + p] = (v >= 0 && (v >> 5) == w) ? (1u << (v & 31)) : 0u;
  b.imgL[(size_t)y * k.pitch + x] = left[p];
  b.imgR[(size_t)y * k.pitch + x] = right[p];
}

cudaError_t launch_ingest(const KParams &k, const Buffers &b, int nf, const uint8_t *left, const uint8_t *right,
                          const float *lidar, cudaStream_t s) {
  dim3 grid((k.W + 31) / 32, (k.H + 7) / 8, nf);
  k_ingest<<<grid, 256, 0, s>>>(k, b, left, right, lidar);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// --------------------------------------------------------------------------
// Census (Sec. IV-A).  Offsets (dx, dy), dx in [-4,4], dy in [-3,3], in raster
// order without the centre; offset k sets bit k.  CS 9x7: the 31 offsets
// before the centre, bit = I(p+o) > I(p-o).  9x7: all 62, bit = I(p+o) > I(p).
// A bit whose samples are not all inside the image is 0.
//
// One CTA computes a 64 x 16 tile of both images.  One thread issues two TMA
// loads of the 96 x 22 byte boxes starting at (x0-16, y0-3): the x start is a
// multiple of 16, and samples outside the image arrive as 0 and are masked
// by the coordinate test on border tiles.
// Census bits of the pixel at tile position (sx, sy): offsets are visited in
// reverse raster order and shifted in, so offset k lands in bit k.  A bit is
// the sign of I(q) - I(p+o) (q = p-o for the centre-symmetric kind, q = p
// otherwise); INTERIOR tiles have every sample inside the image, elsewhere a
// bit with a sample outside is cleared.
template <bool FULL, bool INTERIOR>
__device__ __forceinline__ uint64_t census_bits(const uint8_t (*T)[kCenBoxW], int sx, int sy, int x, int y, int W,
                                                int H) {
  uint64_t c = 0;
  const int centre = T[sy][sx];
#pragma unroll
  for (int dy = 3; dy >= -3; --dy) {
#pragma unroll
    for (int dx = 4; dx >= -4; --dx) {
      if (dx == 0 && dy == 0) continue;
      if (!FULL && (dy > 0 || (dy == 0 && dx > 0))) continue;   // the half before the centre
      const int a = T[sy + dy][sx + dx];
      const int bq = FULL ? centre : (int)T[sy - dy][sx - dx];
      uint32_t bit = (uint32_t)(bq - a) >> 31;                 // a > bq
      if (!INTERIOR) {
        bool in = (unsigned)(x + dx) < (unsigned)W && (unsigned)(y + dy) < (unsigned)H;
        if (!FULL) in = in && (unsigned)(x - dx) < (unsigned)W && (unsigned)(y - dy) < (unsigned)H;
        bit = in ? bit : 0u;
      }
      c = c + c + bit;
    }
  }
  return c;
}

template <bool FULL>
__global__ void __launch_bounds__(256) k_census(KParams k, Buffers b0, const __grid_constant__ CUtensorMap mapL,
                                                const __grid_constant__ CUtensorMap mapR) {
  const int f = blockIdx.z;
  const Buffers b = frame_view(k, b0, f);
  // each box starts on a 128-byte boundary, as cp.async.bulk.tensor requires
  constexpr int kBoxBytes = (kCenBoxH * kCenBoxW + 127) / 128 * 128;
  __shared__ alignas(128) uint8_t tiles[2 * kBoxBytes];
  __shared__ alignas(8) uint64_t bar;
  const int x0 = blockIdx.x * kCenTileW, y0 = blockIdx.y * kCenTileH;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, 2u * kCenBoxW * kCenBoxH);
    tma_load_3d(tiles, &mapL, x0 - 16, y0 - 3, f, &bar);
    tma_load_3d(tiles + kBoxBytes, &mapR, x0 - 16, y0 - 3, f, &bar);
  }
  if (!mbar_wait_bounded(&bar, 0, kWaitLimit)) {
    set_error(b.err, kErrTimeout);
    mbar_wait_bounded(&bar, 0, kWaitLimit);   // give the copies in flight a second chance
    return;
  }
  const bool interior = x0 >= 4 && x0 + kCenTileW + 4 <= k.W && y0 >= 3 && y0 + kCenTileH + 3 <= k.H;
  const int tx = threadIdx.x & 63;
  const int x = x0 + tx;
  for (int r = threadIdx.x >> 6; r < kCenTileH; r += 4) {
    const int y = y0 + r;
    if (x >= k.W || y >= k.H) continue;
    const int sx = tx + 16, sy = r + 3;
    const size_t p = (size_t)y * k.W + x;
#pragma unroll
    for (int img = 0; img < 2; ++img) {
      const uint8_t(*T)[kCenBoxW] = reinterpret_cast<const uint8_t(*)[kCenBoxW]>(tiles + img * kBoxBytes);
      const uint64_t c = interior ? census_bits<FULL, true>(T, sx, sy, x, y, k.W, k.H)
                                  : census_bits<FULL, false>(T, sx, sy, x, y, k.W, k.H);
      if (FULL)
        static_cast<uint64_t *>(img ? b.censR : b.censL)[p] = c;
      else
        static_cast<uint32_t *>(img ? b.censR : b.censL)[p] = (uint32_t)c;
    }
  }
}

cudaError_t launch_census(const KParams &k, const Buffers &b, int nf, const void *tmaL, const void *tmaR,
                          cudaStream_t s) {
  dim3 grid((k.W + kCenTileW - 1) / kCenTileW, (k.H + kCenTileH - 1) / kCenTileH, nf);
  const CUtensorMap &mL = *static_cast<const CUtensorMap *>(tmaL);
  const CUtensorMap &mR = *static_cast<const CUtensorMap *>(tmaR);
  if (k.census == 1)
    k_census<true><<<grid, 256, 0, s>>>(k, b, mL, mR);
  else
    k_census<false><<<grid, 256, 0, s>>>(k, b, mL, mR);
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

int make_image_tmap(void *tmap_out, const uint8_t *base, int W, int H, int pitch, int frames, int box_w,
                    int box_h) {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || ptr == nullptr)
      return -1;
    fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)frames};
  cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)pitch * H};
  cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(static_cast<CUtensorMap *>(tmap_out), CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
                  const_cast<uint8_t *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

// --------------------------------------------------------------------------
// Separable box-OR of presence masks: dst[w][y][x] = OR of src[w][y'][x'] over
// |x'-x| <= r, |y'-y| <= r inside the image.  The OR over a clipped rectangle
// is the OR (over rows) of the ORs along each row, so a row pass followed by
// a column pass is exact.  Each pass builds a doubling table in shared memory
// (level j holds the OR of 2^j consecutive words); OR being idempotent, the
// window of L = 2r+1 words is the OR of two level-k entries (2^k <= L < 2^(k+1))
// that overlap: k + 1 ORs per word instead of L.
constexpr int kBoxRowTile = 256;

__device__ __forceinline__ int floor_log2(int v) { return 31 - __clz(v); }

__global__ void __launch_bounds__(kBoxRowTile) k_boxor_rows(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                           int W, int H, int r) {
  extern __shared__ uint32_t seg[];            // two buffers of n words
  const int y = blockIdx.y, w = blockIdx.z;
  const size_t base = ((size_t)w * H + y) * W;
  const int x0 = blockIdx.x * kBoxRowTile;
  const int n = kBoxRowTile + 2 * r;
  uint32_t *A = seg, *B = seg + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int x = x0 - r + i;
    A[i] = (x >= 0 && x < W) ? src[base + x] : 0u;
  }
  const int L = 2 * r + 1, k = floor_log2(L);
  for (int j = 0; j < k; ++j) {
    __syncthreads();
    const int s = 1 << j;
    for (int i = threadIdx.x; i + s < n; i += blockDim.x) B[i] = A[i] | A[i + s];
    __syncthreads();
    uint32_t *t = A;
    A = B;
    B = t;
  }
  __syncthreads();
  const int x = x0 + threadIdx.x;
  if (x >= W) return;
  // window [threadIdx.x, threadIdx.x + L - 1] of the segment
  dst[base + x] = A[threadIdx.x] | A[threadIdx.x + L - (1 << k)];
}

constexpr int kBoxColW = 32, kBoxColH = 64;

__global__ void __launch_bounds__(256) k_boxor_cols(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                   int W, int H, int r) {
  extern __shared__ uint32_t blk[];            // two buffers of [(kBoxColH + 2r)][kBoxColW]
  const int w = blockIdx.z;
  const size_t plane = (size_t)w * H * W;
  const int x0 = blockIdx.x * kBoxColW, y0 = blockIdx.y * kBoxColH;
  const int rows = kBoxColH + 2 * r;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  uint32_t *A = blk, *B = blk + rows * kBoxColW;
  for (int i = ty; i < rows; i += 8) {
    const int yy = y0 - r + i, x = x0 + tx;
    A[i * kBoxColW + tx] = (yy >= 0 && yy < H && x < W) ? src[plane + (size_t)yy * W + x] : 0u;
  }
  const int L = 2 * r + 1, k = floor_log2(L);
  for (int j = 0; j < k; ++j) {
    __syncthreads();
    const int s = 1 << j;
    for (int i = ty; i + s < rows; i += 8) B[i * kBoxColW + tx] = A[i * kBoxColW + tx] | A[(i + s) * kBoxColW + tx];
    __syncthreads();
    uint32_t *t = A;
    A = B;
    B = t;
  }
  __syncthreads();
  const int x = x0 + tx;
  if (x >= W) return;
  const int off = L - (1 << k);
  for (int oy = ty; oy < kBoxColH; oy += 8) {
    const int y = y0 + oy;
    if (y >= H) break;
    dst[plane + (size_t)y * W + x] = A[oy * kBoxColW + tx] | A[(oy + off) * kBoxColW + tx];
  }
}

cudaError_t launch_boxor(const KParams &k, int nf, const uint32_t *src, uint32_t *tmp, uint32_t *dst, int radius,
                         cudaStream_t s) {
  // frames and mask words are contiguous planes: plane z = f * MW + w
  dim3 g1((k.W + kBoxRowTile - 1) / kBoxRowTile, k.H, nf * k.MW);
  size_t sm1 = 2 * (size_t)(kBoxRowTile + 2 * radius) * sizeof(uint32_t);
  k_boxor_rows<<<g1, kBoxRowTile, sm1, s>>>(src, tmp, k.W, k.H, radius);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 g2((k.W + kBoxColW - 1) / kBoxColW, (k.H + kBoxColH - 1) / kBoxColH, nf * k.MW);
  size_t sm2 = 2 * (size_t)(kBoxColH + 2 * radius) * kBoxColW * sizeof(uint32_t);
  if (sm2 > 48 * 1024) {
    e = cudaFuncSetAttribute(k_boxor_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    if (e != cudaSuccess) return e;
  }
  k_boxor_cols<<<g2, 256, sm2, s>>>(tmp, dst, k.W, k.H, radius);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Semidensification, Eq. 5 (Sec. IV-B).  The candidates of pixel p are the
// distinct valid d-bar_q, q in the (2rs+1)^2 window: exactly the set bits of
// the box-ORed presence mask.  Visiting them in increasing d and keeping the
// first strict minimum of H(p, d) gives the smallest H with ties to the
// smaller disparity.  d-hat = that d if min H < ts, else d-bar_p.
template <typename CT>
__global__ void __launch_bounds__(256) k_semidense(KParams k, Buffers b0) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= k.W || y >= k.H) return;
  const Buffers b = frame_view(k, b0, blockIdx.z);
  const size_t p = (size_t)y * k.W + x;
  const size_t plane = (size_t)k.W * k.H;
  const CT *cl = static_cast<const CT *>(b.censL);
  const CT *cr = static_cast<const CT *>(b.censR);
  const CT c = cl[p];
  int best_h = 0x7fffffff, best_d = -1;
  for (int w = 0; w < k.MW && best_h > 0; ++w) {
    uint32_t m = b.boxS[w * plane + p];
    while (m != 0u) {
      const int d = w * 32 + __ffs(m) - 1;
      m &= m - 1u;
      const int h = (x >= d) ? __popcll((uint64_t)(c ^ cr[p - d])) : k.nbits;
      if (h < best_h) {
        best_h = h;
        best_d = d;
        if (h == 0) break;
      }
    }
  }
  b.dhat[p] = (best_d >= 0 && best_h < k.ts) ? (int16_t)best_d : b.dbar[p];
}

cudaError_t launch_semidense(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  dim3 grid((k.W + 31) / 32, (k.H + 7) / 8, nf);
  if (k.census == 1)
    k_semidense<uint64_t><<<grid, 256, 0, s>>>(k, b);
  else
    k_semidense<uint32_t><<<grid, 256, 0, s>>>(k, b);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Joint cost C-bar (Eq. 4).  H(p,d) = popcount(cL(x,y) ^ cR(x-d,y)), or the
// number of census bits where x - d < 0.  Where the prior (d-hat, or d-bar
// for DSGM) is invalid C-bar = H; otherwise
//   C-bar = floor(((b-a) H + a q + floor(b/2)) / b),  q = 0 / q1 / q2 for
// |d - prior| = 0 / 1 / > 1, looked up in a table built on the host.
// A CTA handles PX pixels of one row (32, 64 or 128, a tuning choice): their
// right-census window is staged in shared memory, the lanes of a warp walk
// the disparities of one pixel, and the CTA's [PX][Dp] cost rows, assembled
// in shared memory, leave as 16-byte stores (cells d >= D hold 0).


template <typename CT>
__device__ __forceinline__ int hamming(CT a, CT b) {
  if constexpr (sizeof(CT) == 4)
    return __popc(a ^ b);
  else
    return __popcll(a ^ b);
}

template <typename CT, int DPL, int PX>
__global__ void __launch_bounds__(256) k_cost(KParams k, Buffers b0, const __grid_constant__ CostTable tab) {
  constexpr int Dp = 32 * DPL;
  __shared__ CT cr_s[PX + Dp];
  __shared__ CT cl_s[PX];
  __shared__ int pd_s[PX];
  __shared__ uint8_t tab_s[4 * 64];
  __shared__ __align__(16) uint8_t out_s[PX * Dp];   // the block's cost rows, [x][d]
  const Buffers b = frame_view(k, b0, blockIdx.z);
  const int x0 = blockIdx.x * PX, y = blockIdx.y, W = k.W;
  const size_t rowp = (size_t)y * W;
  const CT *cl = static_cast<const CT *>(b.censL) + rowp;
  const CT *cr = static_cast<const CT *>(b.censR) + rowp;
  const int16_t *prior = (k.semidense ? b.dhat : b.dbar) + rowp;
  const int base = x0 - (Dp - 1);               // cr_s[i] = cR(base + i)
  for (int i = threadIdx.x; i < PX + Dp - 1; i += blockDim.x) {
    const int xx = base + i;
    cr_s[i] = (xx >= 0 && xx < W) ? cr[xx] : (CT)0;
  }
  if (threadIdx.x < PX) {
    const int xx = x0 + threadIdx.x;
    const int pd = xx < W ? prior[xx] : -1;
    cl_s[threadIdx.x] = xx < W ? cl[xx] : (CT)0;
    pd_s[threadIdx.x] = pd;
  }
  for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x) tab_s[i] = (&tab.v[0][0])[i];
  __syncthreads();
  // lanes walk disparities (d = lane + 32 j): the right-census reads of a warp
  // are consecutive words, free of bank conflicts
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int npx = min(PX, W - x0);
  // warp-uniform fast path: every d of the pixel has x - d >= 0, all cells are
  // real disparities, and without a prior C-bar = H (no table)
  const bool inner = x0 >= Dp - 1 && k.D == Dp;
  for (int px = warp; px < npx; px += 8) {
    const int x = x0 + px;
    const CT c = cl_s[px];
    const int pd = pd_s[px];
    if (inner && pd < 0) {
#pragma unroll
      for (int j = 0; j < DPL; ++j) {
        const int d = lane + 32 * j;
        out_s[px * Dp + d] = (uint8_t)hamming<CT>(c, cr_s[px - d + Dp - 1]);
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < DPL; ++j) {
      const int d = lane + 32 * j;
      const int h = (x >= d) ? hamming<CT>(c, cr_s[px - d + Dp - 1]) : k.nbits;
      const int cls = pd < 0 ? 3 : min(abs(d - pd), 2);
      out_s[px * Dp + d] = d < k.D ? tab_s[cls * 64 + h] : (uint8_t)0;
    }
  }
  __syncthreads();
  // the block's [npx][Dp] bytes are contiguous in the cost volume: 16-byte stores
  uint4 *dst = reinterpret_cast<uint4 *>(b.cost + (rowp + x0) * Dp);
  const uint4 *src = reinterpret_cast<const uint4 *>(out_s);
  const int nvec = npx * Dp / 16;
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = src[i];
}

template <typename CT, int PX>
static void launch_cost_px(const KParams &k, const Buffers &b, int nf, const CostTable &tab, cudaStream_t s) {
  dim3 grid((k.W + PX - 1) / PX, k.H, nf);
  switch (k.DPL) {
    case 2: k_cost<CT, 2, PX><<<grid, 256, 0, s>>>(k, b, tab); break;
    case 4: k_cost<CT, 4, PX><<<grid, 256, 0, s>>>(k, b, tab); break;
    case 6: k_cost<CT, 6, PX><<<grid, 256, 0, s>>>(k, b, tab); break;
    default: k_cost<CT, 8, PX><<<grid, 256, 0, s>>>(k, b, tab); break;
  }
}

// pixels per CTA from the context's tuning (32, 64 or 128)
template <typename CT>
static void launch_cost_t(const KParams &k, const Buffers &b, int nf, const CostTable &tab, cudaStream_t s) {
  switch (k.cost_px) {
    case 32: launch_cost_px<CT, 32>(k, b, nf, tab, s); break;
    case 64: launch_cost_px<CT, 64>(k, b, nf, tab, s); break;
    default: launch_cost_px<CT, 128>(k, b, nf, tab, s); break;
  }
}

cudaError_t launch_cost(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  const CostTable tab = cost_table(k);
  if (k.census == 1)
    launch_cost_t<uint64_t>(k, b, nf, tab, s);
  else
    launch_cost_t<uint32_t>(k, b, nf, tab, s);
  return cudaGetLastError();
}

}  // namespace sgmf
