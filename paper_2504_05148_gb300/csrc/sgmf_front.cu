// sgmf_front.cu -- the stages before aggregation (sm_103a):
//   k_ingest      sparse LiDAR map d-bar + pitched image copies
//   k_census      9x7 census of both images, windows staged in shared memory by TMA
//   k_boxor_*     OR of the presence masks over (2r+1)^2 windows, both radii
//   k_semidense   Eq. 5
//   k_cost        Hamming cost + DDC, Eq. 4, materialised as uint8 [H][W][Dp]
#include <cuda.h>
#include <cstdint>

#include "sgmf_cost.cuh"
#include "sgmf_internal.cuh"

namespace sgmf {

// --------------------------------------------------------------------------
// d-bar (Sec. IV: integer sparse disparity aligned with the left view).
// A LiDAR value f becomes rint(f) (round half to even) when f is finite,
// f > 0 and rint(f) <= D-1; everything else is invalid (-1).  (The presence
// masks, bit d-bar of a pixel, are formed inside the box-OR.)  The images are copied into pitched
// buffers whose rows start on 16-byte boundaries, as TMA requires.
__global__ void __launch_bounds__(256) k_ingest(KParams k, Buffers b0, const uint8_t *__restrict__ left,
                                                const uint8_t *__restrict__ right,
                                                const float *__restrict__ lidar) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= k.W || y >= k.H) return;
  const int f = blockIdx.z;
  const Buffers b = frame_view(k, b0, f);
  if (gated_off(b.gate, k.gate_run)) return;
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
  b.imgL[(size_t)y * k.pitch + x] = left[p];
  b.imgR[(size_t)y * k.pitch + x] = right[p];
}

// d-bar of one LiDAR sample (0 = no return, non-finite or beyond D-1: -1)
__device__ __forceinline__ int lidar_dbar(float f, int D) {
  if (isfinite(f) && f > 0.0f) {
    const float r = rintf(f);
    if (r <= (float)(D - 1)) return (int)r;
  }
  return -1;
}

// The same for even W, four pixels a thread: with y W even, the LiDAR row
// is read as 8-byte pairs, the image rows as 2-byte pairs, d-bar written as
// 4-byte pairs and the pitched rows as 4-byte words (pitch % 16 == 0).
__global__ void __launch_bounds__(256) k_ingest4(KParams k, Buffers b0, const uint8_t *__restrict__ left,
                                                 const uint8_t *__restrict__ right, const float *__restrict__ lidar) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x = blockIdx.x * 128 + 4 * lane, y = blockIdx.y * 8 + warp;
  if (x >= k.W || y >= k.H) return;
  const int f = blockIdx.z;
  const Buffers b = frame_view(k, b0, f);
  if (gated_off(b.gate, k.gate_run)) return;
  const size_t fo = (size_t)f * frame_px(k), p = (size_t)y * k.W + x;
  left += fo;
  right += fo;
  if (lidar != nullptr) lidar += fo;
  if (x + 3 < k.W) {
    int v[4] = {-1, -1, -1, -1};
    if (lidar != nullptr) {
      const float2 l0 = *reinterpret_cast<const float2 *>(lidar + p);
      const float2 l1 = *reinterpret_cast<const float2 *>(lidar + p + 2);
      v[0] = lidar_dbar(l0.x, k.D), v[1] = lidar_dbar(l0.y, k.D);
      v[2] = lidar_dbar(l1.x, k.D), v[3] = lidar_dbar(l1.y, k.D);
    }
    uint32_t *db = reinterpret_cast<uint32_t *>(b.dbar + p);
    db[0] = (uint32_t)(uint16_t)v[0] | ((uint32_t)(uint16_t)v[1] << 16);
    db[1] = (uint32_t)(uint16_t)v[2] | ((uint32_t)(uint16_t)v[3] << 16);
    const uint16_t *l2 = reinterpret_cast<const uint16_t *>(left + p);
    const uint16_t *r2 = reinterpret_cast<const uint16_t *>(right + p);
    *reinterpret_cast<uint32_t *>(b.imgL + (size_t)y * k.pitch + x) = (uint32_t)l2[0] | ((uint32_t)l2[1] << 16);
    *reinterpret_cast<uint32_t *>(b.imgR + (size_t)y * k.pitch + x) = (uint32_t)r2[0] | ((uint32_t)r2[1] << 16);
  } else {
    for (int u = 0; x + u < k.W; ++u) {
      b.dbar[p + u] = (int16_t)(lidar != nullptr ? lidar_dbar(lidar[p + u], k.D) : -1);
      b.imgL[(size_t)y * k.pitch + x + u] = left[p + u];
      b.imgR[(size_t)y * k.pitch + x + u] = right[p + u];
    }
  }
}

cudaError_t launch_ingest(const KParams &k, const Buffers &b, int nf, const uint8_t *left, const uint8_t *right,
                          const float *lidar, cudaStream_t s) {
  // the four-pixel form needs even rows and 8-byte aligned inputs
  const bool four = k.W % 2 == 0 && reinterpret_cast<uintptr_t>(left) % 2 == 0 &&
                    reinterpret_cast<uintptr_t>(right) % 2 == 0 && reinterpret_cast<uintptr_t>(lidar) % 8 == 0;
  if (four) {
    dim3 grid((k.W + 127) / 128, (k.H + 7) / 8, nf);
    k_ingest4<<<grid, 256, 0, s>>>(k, b, left, right, lidar);
  } else {
    dim3 grid((k.W + 31) / 32, (k.H + 7) / 8, nf);
    k_ingest<<<grid, 256, 0, s>>>(k, b, left, right, lidar);
  }
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

// The centre-symmetric census of four horizontally adjacent pixels of an
// interior tile at once, four byte lanes per 32-bit word.  For each offset
// the four pixels' samples I(p+o) and I(p-o) are four consecutive bytes of a
// staged row (byte permutes of three aligned words per row); the per-byte
// unsigned comparison is made with ordinary integer operations: with H the
// bytes' high bits, (b | H) - (a & ~H) borrows across no byte and its high
// bit says low(b) >= low(a), so b >= a is (b & ~a) | (~(a ^ b) & that) on the
// high bits, and a > b its complement.  The offsets' bits are shifted into
// four accumulators of eight offsets each (one bit per byte lane per
// offset), which a byte transpose turns into the four descriptors.
__device__ __forceinline__ uint32_t bytes_gt(uint32_t a, uint32_t b) {
  constexpr uint32_t H = 0x80808080u;
  const uint32_t d = (b | H) - (a & ~H);
  const uint32_t ge = (b & ~a) | (~(a ^ b) & d);
  return ~ge & H;   // high bit of byte j: a_j > b_j
}

// bytes off .. off + 3 of the 12 bytes w[0..2] (off in 0..8, a constant)
__device__ __forceinline__ uint32_t bytes_at(const uint32_t (&w)[3], int off) {
  const int i = off >> 2, sh = off & 3;
  return sh == 0 ? w[i] : __byte_perm(w[i], w[i + 1], 0x3210u + 0x1111u * (uint32_t)sh);
}

// descriptors of the tile pixels (sx .. sx + 3, sy) of one staged box
__device__ __forceinline__ void census_cs4(const uint8_t *box, int sx, int sy, uint32_t (&desc)[4]) {
  uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int dy = 0; dy >= -3; --dy) {
    const uint32_t *ra = reinterpret_cast<const uint32_t *>(box + (sy + dy) * kCenBoxW + sx - 4);
    const uint32_t *rb = reinterpret_cast<const uint32_t *>(box + (sy - dy) * kCenBoxW + sx - 4);
    const uint32_t A[3] = {ra[0], ra[1], ra[2]}, B[3] = {rb[0], rb[1], rb[2]};
#pragma unroll
    for (int dx = 4; dx >= -4; --dx) {
      if (dy == 0 && dx >= 0) continue;   // the half before the centre
      const int kbit = (dy + 3) * 9 + (dx + 4);   // offsets visited in decreasing k
      const uint32_t gt = bytes_gt(bytes_at(A, dx + 4), bytes_at(B, 4 - dx));
      acc[kbit >> 3] = acc[kbit >> 3] * 2u + (gt >> 7);
    }
  }
  const uint32_t lo = __byte_perm(acc[0], acc[1], 0x5140), hi = __byte_perm(acc[2], acc[3], 0x5140);
  const uint32_t lo2 = __byte_perm(acc[0], acc[1], 0x7362), hi2 = __byte_perm(acc[2], acc[3], 0x7362);
  desc[0] = __byte_perm(lo, hi, 0x5410);
  desc[1] = __byte_perm(lo, hi, 0x7632);
  desc[2] = __byte_perm(lo2, hi2, 0x5410);
  desc[3] = __byte_perm(lo2, hi2, 0x7632);
}

// b0 holds the buffers of the launch's first frame, which is frame zoff of
// the tensor maps (their third coordinate)
template <bool FULL>
__global__ void __launch_bounds__(256) k_census(KParams k, Buffers b0, int zoff,
                                                const __grid_constant__ CUtensorMap mapL,
                                                const __grid_constant__ CUtensorMap mapR) {
  const int f = blockIdx.z;
  const Buffers b = frame_view(k, b0, f);
  if (gated_off(b.gate, k.gate_run)) return;
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
    tma_load_3d(tiles, &mapL, x0 - 16, y0 - 3, zoff + f, &bar);
    tma_load_3d(tiles + kBoxBytes, &mapR, x0 - 16, y0 - 3, zoff + f, &bar);
  }
  if (!mbar_wait_bounded(&bar, 0, k.wait_census)) {
    set_error(b.err, kErrTimeout);
    mbar_wait_bounded(&bar, 0, kWaitLimit);   // the copies in flight land before the CTA exits
    return;
  }
  const bool interior = x0 >= 4 && x0 + kCenTileW + 4 <= k.W && y0 >= 3 && y0 + kCenTileH + 3 <= k.H;
  if (!FULL && interior) {
    // four pixels a thread: 16 threads a tile row, 16 rows
    static_assert(kCenTileW == 64 && kCenTileH == 16, "census_cs4 covers the tile with 256 threads");
    const int g = threadIdx.x & 15, r = threadIdx.x >> 4;
    const int x = x0 + 4 * g, y = y0 + r;
    const size_t p = (size_t)y * k.W + x;
#pragma unroll
    for (int img = 0; img < 2; ++img) {
      uint32_t d[4];
      census_cs4(tiles + img * kBoxBytes, 4 * g + 16, r + 3, d);
      uint32_t *o = static_cast<uint32_t *>(img ? b.censR : b.censL) + p;
#pragma unroll
      for (int u = 0; u < 4; ++u) o[u] = d[u];
    }
    return;
  }
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

cudaError_t launch_census(const KParams &k, const Buffers &b, int nf, int zoff, const void *tmaL, const void *tmaR,
                          cudaStream_t s) {
  dim3 grid((k.W + kCenTileW - 1) / kCenTileW, (k.H + kCenTileH - 1) / kCenTileH, nf);
  const CUtensorMap &mL = *static_cast<const CUtensorMap *>(tmaL);
  const CUtensorMap &mR = *static_cast<const CUtensorMap *>(tmaR);
  if (k.census == 1)
    k_census<true><<<grid, 256, 0, s>>>(k, b, zoff, mL, mR);
  else
    k_census<false><<<grid, 256, 0, s>>>(k, b, zoff, mL, mR);
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
// Box-OR of the presence masks (the windows of Eq. 5 and Eq. 6):
// box[w][y][x] = OR, over the pixels (x', y') with |x'-x| <= r, |y'-y| <= r
// inside the image whose sparse disparity d = disp(x', y') lies in [0, D),
// of bit d & 31 of word d >> 5.  The OR over a clipped square is the OR over
// its rows of the ORs along each row, so a row pass and a column pass make
// it exactly.  Both radii (r_s of Eq. 5, r_c of Eq. 6) come out of one row
// pass; the column pass runs for r_s only.  The r_c row ORs stay as they are
// (in boxC): Eq. 6 needs its LiDAR term only at pixels whose stereo term
// fails, and the check kernel ORs those pixels' 2 r_c + 1 rows itself.
//
// Row pass, from the sparse map itself: a warp owns 32 consecutive pixels of
// one row and visits the valid pixels of [x0 - R, x0 + 31 + R] (R the larger
// radius) 32 at a time: a ballot finds them, a shuffle hands out each one's
// disparity, and every lane ORs its bit into the words of the radii that
// reach it.  The work follows the number of valid pixels, not r.
template <int MW>
__global__ void __launch_bounds__(256) k_boxor_rows(const int16_t *__restrict__ disp, uint32_t *__restrict__ tmpS,
                                                   uint32_t *__restrict__ tmpC, int W, int H, int D, int rs,
                                                   int rc, const int *gate, int run) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y = blockIdx.y * 8 + warp;
  if (y >= H) return;                          // warps are independent: no block barrier
  const int f = blockIdx.z;
  if (gated_off(gate ? gate + f : nullptr, run)) return;
  const int x0 = blockIdx.x * 32, x = x0 + lane;
  const int16_t *row = disp + ((size_t)f * H + y) * W;
  const int R = max(rs, rc);                   // an unwanted radius is -1: no pixel is that close
  uint32_t aS[MW], aC[MW];
#pragma unroll
  for (int w = 0; w < MW; ++w) aS[w] = aC[w] = 0u;
  for (int base = x0 - R; base <= x0 + 31 + R; base += 32) {
    const int xs = base + lane;
    const int d = (xs >= 0 && xs < W) ? (int)row[xs] : -1;
    unsigned m = __ballot_sync(0xffffffffu, d >= 0 && d < D);
    while (m != 0u) {
      const int j = __ffs(m) - 1;
      m &= m - 1u;
      const int dp = __shfl_sync(0xffffffffu, d, j);
      const int dx = abs(base + j - x);
      const uint32_t bc = dx <= rc ? 1u << (dp & 31) : 0u, bs = dx <= rs ? 1u << (dp & 31) : 0u;
      // the point's word plane is the same for the whole warp: a uniform branch
      switch (dp >> 5) {
#define SGMF_BOX_ACC(w)      \
  case w:                    \
    if constexpr (w < MW) {  \
      aC[w] |= bc;           \
      aS[w] |= bs;           \
    }                        \
    break;
        SGMF_BOX_ACC(0) SGMF_BOX_ACC(1) SGMF_BOX_ACC(2) SGMF_BOX_ACC(3)
        SGMF_BOX_ACC(4) SGMF_BOX_ACC(5) SGMF_BOX_ACC(6) SGMF_BOX_ACC(7)
#undef SGMF_BOX_ACC
        default: break;
      }
    }
  }
  if (x >= W) return;
  const size_t plane = (size_t)H * W, o = (size_t)f * MW * plane + (size_t)y * W + x;
#pragma unroll
  for (int w = 0; w < MW; ++w) {
    if (rs >= 0) tmpS[o + w * plane] = aS[w];
    if (rc >= 0) tmpC[o + w * plane] = aC[w];
  }
}

// Column pass (van Herk / Gil-Werman): with the rows cut into blocks of
// L = 2r + 1, the window [u, u + 2r] is the suffix OR of u's block from u
// together with the prefix OR of (u + 2r)'s block up to u + 2r, so every
// output costs O(1) whatever r.  A lane owns one column, the 32 lanes of a
// warp on consecutive x (every load is one coalesced row segment), and
// streams kColSeg output rows from the kColSeg + 2r input rows above and
// below them, each read once, loads kColChunk rows ahead.  Segments are
// kColSeg rows, or down to kColSegMin for grids that would not fill the GPU
// (few frames a call), whose CTAs re-read more halo rows but run in parallel.  It keeps two
// blocks in shared memory: the raw rows of the block being read (its prefix
// OR runs in a register) and, once a block is complete, its suffix ORs in
// place.  Output i = u - 2r, read when row u arrives, lies in u's block (u at
// the block's end, i at its start) or in the block before, so two buffers
// alternating by block are enough.
constexpr int kColSeg = 128, kColSegMin = 32, kColChunk = 8;

__host__ __device__ constexpr int boxor_col_smem(int r) { return 2 * (2 * r + 1) * 32 * 4; }

__global__ void __launch_bounds__(32) k_boxor_cols(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                  int W, int H, int MW, int r, int seg, const int *gate, int run) {
  extern __shared__ uint32_t colbuf[];         // [2][L][32]: the two blocks, one word per lane
  const int lane = threadIdx.x;
  const int f = blockIdx.z / MW, w = blockIdx.z % MW;
  if (gated_off(gate ? gate + f : nullptr, run)) return;
  const size_t base = ((size_t)f * MW + w) * H * W;
  const int x = blockIdx.x * 32 + lane, y0 = blockIdx.y * seg;
  const int L = 2 * r + 1, T = min(seg, H - y0), n = T + 2 * r, ylo = y0 - r;
  const bool live = x < W;
  // lanes past the image's right edge read its last column and store nothing
  const uint32_t *col = src + base + min(x, W - 1);
  uint32_t *o = dst + base + min(x, W - 1) + (size_t)y0 * W;
  // input row u is image row ylo + u, zero outside the image
  auto load = [&](int u) -> uint32_t {
    const int y = ylo + u;
    return u < n && y >= 0 && y < H ? col[(size_t)y * W] : 0u;
  };
  uint32_t nxt[kColChunk];
#pragma unroll
  for (int k = 0; k < kColChunk; ++k) nxt[k] = load(k);
  uint32_t pre = 0u;                           // prefix OR of u's block up to u
  int p = 0, kb = 0;                           // u's position in its block, the block's buffer
  for (int u0 = 0; u0 < n; u0 += kColChunk) {
    uint32_t cur[kColChunk];
#pragma unroll
    for (int k = 0; k < kColChunk; ++k) {
      cur[k] = nxt[k];
      nxt[k] = load(u0 + kColChunk + k);
    }
#pragma unroll
    for (int k = 0; k < kColChunk; ++k) {
      const int u = u0 + k;
      if (u >= n) break;
      uint32_t *b = colbuf + lane + (kb ? L * 32 : 0), *prev = colbuf + lane + (kb ? 0 : L * 32);
      if (p == 0) pre = 0u;
      pre |= cur[k];
      b[p * 32] = cur[k];
      if (p == L - 1) {
        // the block is complete: its suffix ORs, in place
        uint32_t sfx = 0u;
#pragma unroll 4
        for (int q = L - 1; q >= 0; --q) {
          sfx |= b[q * 32];
          b[q * 32] = sfx;
        }
      }
      if (u >= 2 * r) {
        // i = u - 2r sits at position p + 1 of the previous block, or at 0 of this one
        const int i = u - 2 * r;
        const uint32_t sfx = p == L - 1 ? b[0] : prev[(p + 1) * 32];
        if (live) o[(size_t)i * W] = sfx | pre;
      }
      if (p == L - 1) {
        p = 0;
        kb ^= 1;
      } else {
        ++p;
      }
    }
  }
}

template <int MW>
static void launch_boxor_rows(const KParams &k, int nf, const int16_t *disp, uint32_t *tS, uint32_t *tC, int rs,
                              int rc, cudaStream_t s, const int *gate) {
  dim3 g((k.W + 31) / 32, (k.H + 7) / 8, nf);
  k_boxor_rows<MW><<<g, 256, 0, s>>>(disp, tS, tC, k.W, k.H, k.D, rs, rc, gate, k.gate_run);
}

// the column pass over nf frames: dst = the (2r+1)-row OR of the row results src
cudaError_t launch_boxor_cols(const KParams &k, int nf, const uint32_t *src, uint32_t *dst, int r, cudaStream_t s,
                              const int *gate) {
  static bool done[64] = {};
  cudaError_t e = once_per_device(done, [](int) {
    return cudaFuncSetAttribute(k_boxor_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, boxor_col_smem(255));
  });
  int sms = 0;
  if (e == cudaSuccess) e = sm_count(&sms);
  if (e != cudaSuccess) return e;
  // the longest segment whose grid still makes about two waves of one-warp
  // CTAs (about 20 resident a SM at r = 20)
  const long ctas_per_seg = (long)((k.W + 31) / 32) * nf * k.MW;
  int seg = kColSeg;
  while (seg > kColSegMin && ctas_per_seg * ((k.H + seg - 1) / seg) < 40L * sms) seg /= 2;
  // y: row segment, z: frame x word plane
  dim3 g((k.W + 31) / 32, (k.H + seg - 1) / seg, nf * k.MW);
  k_boxor_cols<<<g, 32, boxor_col_smem(r), s>>>(src, dst, k.W, k.H, k.MW, r, seg, gate, k.gate_run);
  return cudaGetLastError();
}

cudaError_t launch_boxor(const KParams &k, int nf, const int16_t *disp, uint32_t *tmp, uint32_t *boxS,
                         uint32_t *boxC, cudaStream_t s, const int *gate) {
  const int rs = boxS != nullptr ? k.rs : -1, rc = boxC != nullptr ? k.rc : -1;
  if (rs < 0 && rc < 0) return cudaSuccess;
  // the row results: r_s into tmp (for the column pass), r_c into boxC itself
  uint32_t *tS = tmp, *tC = boxC;
  switch (k.MW) {
    case 2: launch_boxor_rows<2>(k, nf, disp, tS, tC, rs, rc, s, gate); break;
    case 4: launch_boxor_rows<4>(k, nf, disp, tS, tC, rs, rc, s, gate); break;
    case 6: launch_boxor_rows<6>(k, nf, disp, tS, tC, rs, rc, s, gate); break;
    case 8: launch_boxor_rows<8>(k, nf, disp, tS, tC, rs, rc, s, gate); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || rs < 0) return e;
  return launch_boxor_cols(k, nf, tS, boxS, rs, s, gate);
}

// --------------------------------------------------------------------------
// Semidensification, Eq. 5 (Sec. IV-B).  The candidates of pixel p are the
// distinct valid d-bar_q, q in the (2rs+1)^2 window: exactly the set bits of
// the box-ORed presence mask.  The smallest key H(p, d) << 9 | d over them is
// the smallest H with ties to the smaller disparity.  d-hat = that d if
// min H < ts, else d-bar_p.
template <typename CT>
__global__ void __launch_bounds__(256) k_semidense(KParams k, Buffers b0) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= k.W || y >= k.H) return;
  const Buffers b = frame_view(k, b0, blockIdx.z);
  if (gated_off(b.gate, k.gate_run)) return;
  const size_t p = (size_t)y * k.W + x;
  const size_t plane = (size_t)k.W * k.H;
  const CT *cl = static_cast<const CT *>(b.censL);
  const CT *cr = static_cast<const CT *>(b.censR);
  const CT c = cl[p];
  // the mask words (MW <= 8), all loads in flight before the first is used
  uint32_t mw[8];
#pragma unroll
  for (int w = 0; w < 8; ++w) mw[w] = w < k.MW ? b.boxS[w * plane + p] : 0u;
  uint32_t best = 0xffffffffu;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    if (w >= k.MW || best < 512u) break;   // H = 0 found: no later candidate wins
    uint32_t m = mw[w];
    while (m != 0u) {
      const int d = w * 32 + __ffs(m) - 1;
      m &= m - 1u;
      const uint32_t h = (x >= d) ? (uint32_t)__popcll((uint64_t)(c ^ cr[p - d])) : (uint32_t)k.nbits;
      best = min(best, h << 9 | (uint32_t)d);
    }
  }
  b.dhat[p] = (best != 0xffffffffu && (int)(best >> 9) < k.ts) ? (int16_t)(best & 511u) : b.dbar[p];
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
// Joint cost C-bar (Eq. 4), with semidensification (Eq. 5) fused in.
// H(p,d) = popcount(cL(x,y) ^ cR(x-d,y)), or the number of census bits where
// x - d < 0.  Where the prior (d-hat, or d-bar for DSGM) is invalid C-bar = H;
// otherwise
//   C-bar = floor(((b-a) H + a q + floor(b/2)) / b),  q = 0 / q1 / q2 for
// |d - prior| = 0 / 1 / > 1, looked up in a table built on the host.
//
// A CTA takes a segment of one row (up to 8 x cost_px pixels, a tuning
// choice: 256, 512 or 1024) and stages the right-census window of the
// segment in shared memory once.  Then (1) one thread per pixel computes
// d-hat of Eq. 5 from the box-ORed mask of its r_s window: the candidates are
// the mask's set bits, each H taken from the staged window; the smallest key
// H << 9 | d over them is the lexicographic (H, d) minimum, with no branch
// per candidate; d-hat = that d if min H < T_s, else d-bar (staging the
// segment's mask words and d-bar with the census window instead was 13 %
// slower: the whole CTA then waits on those loads); (2) a warp takes P = 4
// consecutive pixels at a time,
// each lane the same DPL disparities of all four: the P + DPL - 1 window
// entries cR(x - d) they need are consecutive and start on a vector boundary
// (x - d0 is a multiple of 4 there), so a lane loads them with a few aligned
// vector loads and indexes them with constants; a lane stores DPL cost bytes
// a pixel, a warp's stores one contiguous row of the cost volume.  (Eight
// pixels a step, for fewer loop and load instructions, ran 14 % slower: the
// registers they need halve the resident warps.)
template <typename CT, int DPL, bool SEMI>
__global__ void __launch_bounds__(256) k_cost_seg(KParams k, Buffers b0, const __grid_constant__ CostTable tab,
                                                  int seg, int nwin) {
  constexpr int Dp = 32 * DPL, P = kCostPix;
  __shared__ uint8_t tab_s[4 * 64];                           // fixed address: LDS [h + const]
  extern __shared__ __align__(16) uint8_t cs_smem[];
  const int segr = (seg + P - 1) / P * P;
  CT *cr_s = reinterpret_cast<CT *>(cs_smem);                 // [nwin]: cr_s[j] = cR(x0 - (Dp - 1) + j)
  CT *cl_s = cr_s + nwin;                                     // [segr]
  int16_t *pd_s = reinterpret_cast<int16_t *>(cl_s + segr);   // the prior of each pixel
  const Buffers b = frame_view(k, b0, blockIdx.z);
  if (gated_off(b.gate, k.gate_run)) return;
  const int x0 = blockIdx.x * seg, y = blockIdx.y, W = k.W;
  const int npx = min(seg, W - x0);
  const int npr = (npx + P - 1) / P * P;
  const size_t rowp = (size_t)y * W;
  const CT *cl = static_cast<const CT *>(b.censL) + rowp;
  const CT *cr = static_cast<const CT *>(b.censR) + rowp;
  const int base = x0 - (Dp - 1);
  // the d-bar and r_s mask words (MW = DPL) of the thread's pixels
  // tid + 256 j, loaded first so that their latency overlaps the staging
  constexpr int PPT = 4;   // pixels a thread takes at most (segments of <= 1024 pixels)
  const size_t plane = (size_t)W * k.H;
  int16_t db_r[PPT];
  uint32_t mw_r[PPT][DPL];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int i = threadIdx.x + 256 * j;
    const size_t p = rowp + x0 + i;
    db_r[j] = i < npx ? b.dbar[p] : (int16_t)-1;
#pragma unroll
    for (int w = 0; w < DPL; ++w) mw_r[j][w] = (SEMI && i < npx) ? b.boxS[w * plane + p] : 0u;
  }
  for (int j = threadIdx.x; j < nwin; j += blockDim.x) {
    const int xx = base + j;
    cr_s[j] = (xx >= 0 && xx < W) ? cr[xx] : (CT)0;
  }
  for (int i = threadIdx.x; i < npr; i += blockDim.x) cl_s[i] = i < npx ? cl[x0 + i] : (CT)0;
  for (int i = threadIdx.x; i < 4 * 64; i += blockDim.x) tab_s[i] = (&tab.v[0][0])[i];
  __syncthreads();
  // (1) the prior of every pixel of the segment
#pragma unroll
  for (int jj = 0; jj < PPT; ++jj) {
    const int i = threadIdx.x + 256 * jj;
    if (i >= npr) break;
    if (i >= npx) {
      pd_s[i] = -1;
      continue;
    }
    const size_t p = rowp + x0 + i;
    const int db = db_r[jj];
    int pd = db;
    if (SEMI) {
      const int x = x0 + i;
      const CT c = cl_s[i];
      // the candidates in rising d; the smallest key H << 9 | d is the
      // smallest H, ties to the smallest d (d < 512, H < 128)
      uint32_t best = 0xffffffffu;
#pragma unroll
      for (int w = 0; w < DPL; ++w) {
        if (best < 512u) break;   // H = 0 found: no later candidate wins
        uint32_t m = mw_r[jj][w];
        while (m != 0u) {
          const int d = w * 32 + __ffs(m) - 1;
          m &= m - 1u;
          const uint32_t h = x >= d ? (uint32_t)hamming<CT>(c, cr_s[i + Dp - 1 - d]) : (uint32_t)k.nbits;
          best = min(best, h << 9 | (uint32_t)d);
        }
      }
      pd = (best != 0xffffffffu && (int)(best >> 9) < k.ts) ? (int)(best & 511u) : db;
      b.dhat[p] = (int16_t)pd;
    }
    pd_s[i] = (int16_t)pd;
  }
  __syncthreads();
  // (2) the cost bytes, four pixels per warp at a time
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint8_t *out = b.cost + (rowp + x0) * Dp + DPL * lane;
  for (int xb = P * warp; xb < npx; xb += P * nwarp) {
    uint32_t o[P][DPL];
    cost_quad<CT, DPL>(cr_s, cl_s, pd_s, xb, x0 + xb, lane, k.D, k.nbits, tab_s, o);
#pragma unroll
    for (int u = 0; u < P; ++u)
      if (xb + u < npx) store_cost_bytes<DPL>(out + (size_t)(xb + u) * Dp, o[u]);
  }
}

template <typename CT, bool SEMI>
static cudaError_t launch_cost_t(const KParams &k, const Buffers &b, int nf, const CostTable &tab, cudaStream_t s) {
  // segments of at most 8 x cost_px pixels (at most 1024: four a thread in the Eq. 5 step), equal lengths
  const int segmax = min(8 * k.cost_px, 1024);
  const int nseg = (k.W + segmax - 1) / segmax, seg = (k.W + nseg - 1) / nseg;
  const int Dp = k.Dp;
  const int segr = (seg + kCostPix - 1) / kCostPix * kCostPix;
  const int nwin = (segr + Dp + 3) / 4 * 4;                 // window entries, 16-byte multiple
  const size_t smem = (size_t)nwin * sizeof(CT) + (size_t)segr * sizeof(CT) + (size_t)segr * 2;
  dim3 grid(nseg, k.H, nf);
  // at most (1024 + 256 + 4) + 1024 u64 entries + the priors: below the 48 KiB default
  if (smem > 48 * 1024) return cudaErrorInvalidConfiguration;
  auto launch = [&](auto kern) -> cudaError_t {
    kern<<<grid, 256, smem, s>>>(k, b, tab, seg, nwin);
    return cudaGetLastError();
  };
  switch (k.DPL) {
    case 2: return launch(k_cost_seg<CT, 2, SEMI>);
    case 4: return launch(k_cost_seg<CT, 4, SEMI>);
    case 6: return launch(k_cost_seg<CT, 6, SEMI>);
    default: return launch(k_cost_seg<CT, 8, SEMI>);
  }
}

cudaError_t launch_cost(const KParams &k, const Buffers &b, int nf, cudaStream_t s) {
  const CostTable tab = cost_table(k);
  if (k.census == 1)
    return k.semidense ? launch_cost_t<uint64_t, true>(k, b, nf, tab, s) : launch_cost_t<uint64_t, false>(k, b, nf, tab, s);
  return k.semidense ? launch_cost_t<uint32_t, true>(k, b, nf, tab, s) : launch_cost_t<uint32_t, false>(k, b, nf, tab, s);
}

}  // namespace sgmf
