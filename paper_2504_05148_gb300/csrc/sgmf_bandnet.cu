// sgmf_bandnet.cu -- the band-proposal network (not in the paper): 3x3
// convolutions with 32 channels at quarter resolution on the fifth-generation
// tensor cores (tcgen05.mma, BF16 operands, FP32 accumulators in tensor
// memory), its gradients, loss, optimiser, and the kernels that turn its
// output into band starts for the banded mode.
//
// A convolution is an implicit GEMM.  Forward: D[p][co] = sum_k A[p][k] B[co][k]
// with k = tap * 32 + ci (tap = ky * 3 + kx), A the im2col rows of 128 output
// pixels and B the weights: M = 128, N = 32, K = 288 = 18 MMAs of K = 16.
// The data gradient is the same GEMM on the output gradient with the weights
// rotated by 180 degrees and transposed; the weight gradient is a GEMM over
// pixels: D[(tap, ci)][co] = sum_p X[p + o_tap][ci] dY[p][co] (M = 288 in three
// tiles of 128, N = 32, K = 128 pixels per step).
//
// Shared-memory operands use the K-major layout without swizzle: 8 x 8
// element core matrices of 128 contiguous bytes (8 rows of 16 bytes); the
// descriptor's leading byte offset is the step between core matrices along
// K, its stride byte offset the step between 8-row groups.  One thread
// issues the MMAs; tcgen05.commit arrives on an mbarrier that every thread
// waits on (bounded), then each warp reads its 32 accumulator rows with
// tcgen05.ld.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sgmf.h"
#include "sgmf_internal.cuh"

namespace sgmf {

// ---- tcgen05 helpers (inline PTX) -------------------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (tensor memory) (+)= A (smem) * B (smem)^T, BF16 in, FP32 accumulate
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive accumulator columns of this warp's 32 lanes: thread t gets lane (taddr.lane + t)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of this architecture; base offset 0, no swizzle
  return d;
}

// instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32 D
constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

constexpr int kBnC = 32;               // channels
constexpr int kBnK = 9 * kBnC;         // 288
constexpr int kBnKChunks = kBnK / 8;   // 36 core-matrix columns
constexpr int kBnB = kBnC * kBnK * 2;  // 18432 bytes: the packed weights

// byte offset of element (row, k) in a K-major core-matrix image with kc core columns
__host__ __device__ __forceinline__ int cm_off(int row, int k, int kc) {
  return ((row >> 3) * kc + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint16_t f2bf(float f) {
  const __nv_bfloat16 b = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t *>(&b);
}
__device__ __forceinline__ float bf2f(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

// ---- weights -> B images ------------------------------------------------------------
// w: bf16 [co][ky][kx][ci].  fwd image: row co, k = tap * 32 + ci.  dgrad
// image (the transposed, rotated kernel): row ci, k = tap' * 32 + co, holding
// w[co][2 - ky'][2 - kx'][ci].
__global__ void k_bn_pack(const uint16_t *__restrict__ w, uint16_t *__restrict__ fwd, uint16_t *__restrict__ dgr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kBnC * kBnK) return;
  const int co = i / kBnK, r = i % kBnK, tap = r / kBnC, ci = r % kBnC;
  const uint16_t v = w[i];
  if (fwd) fwd[cm_off(co, tap * kBnC + ci, kBnKChunks) / 2] = v;
  if (dgr) dgr[cm_off(ci, (8 - tap) * kBnC + co, kBnKChunks) / 2] = v;
}

// ---- forward / data-gradient convolution ------------------------------------------------
struct BnConvArgs {
  int n, h, w;
  const uint16_t *x;        // bf16 [n][h][w][32]
  const uint4 *packed;      // B image (kBnB bytes)
  const float *bias;        // [32] or null
  int relu;
  const uint16_t *mask;     // bf16 activations: zero the output where mask <= 0 (ReLU gradient), or null
  uint16_t *y;              // bf16 [n][h][w][32] or null
  float *yf;                // f32 [n][h][w][32] or null
  int *err;
};

// One CTA walks `tiles` tiles of 128 consecutive output pixels of one image
// row.  The three input rows of a tile are staged once, split into the four
// 8-channel chunks: Xs[ky][chunk][130 pixels][8 channels] (16 bytes per pixel
// and chunk).  For tap (ky, kx) and channels 16h .. 16h + 15 the A operand is
// then the staged rows themselves, shifted by kx pixels: its core matrices
// (8 pixels x 16 bytes) are contiguous 128-byte blocks, the next 8 rows 128
// bytes further (stride byte offset) and the second chunk one chunk plane
// further (leading byte offset).  No im2col copy: 18 MMAs read the same
// ~25 KB of staged input through different descriptor start addresses.
constexpr int kCvM = 128, kCvPix = kCvM + 2;           // output pixels, staged pixels per row
constexpr int kCvPlane = kCvPix * 16;                  // bytes of one chunk plane (2080)
constexpr int kCvX = 3 * 4 * kCvPlane;                 // 24960 bytes of staged input
constexpr int kCvSmem = kCvX + kBnB + 16;

__global__ void __launch_bounds__(128) k_bn_conv(const __grid_constant__ BnConvArgs a, int tiles) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t *Xs = sm;
  uint8_t *Bs = sm + kCvX;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kCvX + kBnB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + kCvX + kBnB + 8);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tmem_alloc(slot, 32);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  {
    // the packed weights, three loads a thread in flight at a time
    constexpr int kPerThread = kBnB / 16 / 128;
    static_assert(kBnB % (16 * 128) == 0 && kPerThread % 3 == 0, "the weights split evenly over the CTA");
#pragma unroll 1
    for (int s0 = 0; s0 < kPerThread; s0 += 3) {
      uint4 wv[3];
#pragma unroll
      for (int s = 0; s < 3; ++s) wv[s] = a.packed[tid + (s0 + s) * 128];
#pragma unroll
      for (int s = 0; s < 3; ++s) reinterpret_cast<uint4 *>(Bs)[tid + (s0 + s) * 128] = wv[s];
    }
  }
  const int tpr = (a.w + kCvM - 1) / kCvM;                   // tiles per image row
  const long long ntile = (long long)a.n * a.h * tpr;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  const uint32_t idesc = idesc_bf16(128, 32);
  // the 16-byte pieces a thread stages: rows y-1, y, y+1, pixels x0-1 ..
  // x0+128, four chunks each; all of a tile's loads are issued together, and
  // the next tile's while this one's MMAs and epilogue run
  constexpr int kPieces = 3 * kCvPix * 4, kPer = (kPieces + 127) / 128;
  auto fetch = [&](long long tile, uint4 (&v)[kPer]) {
    const int x0 = (int)(tile % tpr) * kCvM;
    const long long row = tile / tpr;                        // img * h + y
    const int y = (int)(row % a.h);
    const long long img = row / a.h;
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int i = tid + s * 128;
      const int j = i & 3, px = (i >> 2) % kCvPix, ky = (i >> 2) / kCvPix;
      const int yy = y + ky - 1, xx = x0 - 1 + px;
      const bool in = i < kPieces && yy >= 0 && yy < a.h && xx >= 0 && xx < a.w;
      v[s] = in ? reinterpret_cast<const uint4 *>(a.x + ((img * a.h + yy) * a.w + xx) * kBnC)[j]
                : make_uint4(0, 0, 0, 0);
    }
  };
  uint4 pf[kPer];
  const long long tile0 = (long long)blockIdx.x * tiles;
  if (tile0 < ntile) fetch(tile0, pf);
  bool ok = true;
  int phase = 0;
  for (int it = 0; it < tiles && ok; ++it) {
    const long long tile = tile0 + it;
    if (tile >= ntile) break;                                // CTA-uniform
    const int tx = (int)(tile % tpr);
    const long long row = tile / tpr;                        // img * h + y
    const int x0 = tx * kCvM;
    // the staged rows as chunk planes
#pragma unroll
    for (int s = 0; s < kPer; ++s) {
      const int i = tid + s * 128;
      if (i < kPieces) {
        const int j = i & 3, px = (i >> 2) % kCvPix, ky = (i >> 2) / kCvPix;
        *reinterpret_cast<uint4 *>(Xs + (ky * 4 + j) * kCvPlane + px * 16) = pf[s];
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t x_0 = smem_u32(Xs), b0 = smem_u32(Bs);
#pragma unroll 1
      for (int t = 0; t < 9; ++t) {
        const int ky = t / 3, kx = t % 3;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t as = x_0 + (ky * 4 + 2 * h) * kCvPlane + kx * 16;
          umma_bf16(tmem, sdesc(as, kCvPlane, 128), sdesc(b0 + (t * 2 + h) * 256, 128, kBnKChunks * 128), idesc,
                    (t > 0 || h > 0) ? 1u : 0u);
        }
      }
      umma_commit(bar);
    }
    if (it + 1 < tiles && tile + 1 < ntile) fetch(tile + 1, pf);
    __syncwarp();
    const bool w_ok = mbar_wait_bounded(bar, (uint32_t)(phase & 1), kWaitLimit);
    ++phase;
    if (!__syncthreads_and(w_ok)) {
      if (tid == 0) set_error(a.err, kErrTimeout);
      mbar_wait_bounded(bar, (uint32_t)((phase - 1) & 1), kWaitLimit);   // MMAs in flight finish first
      ok = false;
      break;
    }
    tc_fence_after();
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
    const int x = x0 + tid;
    if (x < a.w) {
      const long long p = row * a.w + x;
      if (a.bias) {
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] += a.bias[c];
      }
      if (a.relu) {
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c], 0.0f);
      }
      if (a.mask) {
        const uint4 *mk = reinterpret_cast<const uint4 *>(a.mask + p * kBnC);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint4 m = mk[j];
          const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t lo = mw[q] & 0xffffu, hi = mw[q] >> 16;
            // bf16 > 0: sign bit clear and not zero
            if (!(lo != 0 && !(lo & 0x8000u))) v[8 * j + 2 * q] = 0.0f;
            if (!(hi != 0 && !(hi & 0x8000u))) v[8 * j + 2 * q + 1] = 0.0f;
          }
        }
      }
      if (a.yf) {
        float4 *o = reinterpret_cast<float4 *>(a.yf + p * kBnC);
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
      }
      if (a.y) {
        uint4 *o = reinterpret_cast<uint4 *>(a.y + p * kBnC);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t u[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            u[q] = (uint32_t)f2bf(v[8 * j + 2 * q]) | ((uint32_t)f2bf(v[8 * j + 2 * q + 1]) << 16);
          o[j] = make_uint4(u[0], u[1], u[2], u[3]);
        }
      }
    }
    // the accumulator and the staged input are reused by the next tile
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

// ---- weight gradient ---------------------------------------------------------------------
// Each CTA reduces `chunks` chunks of 128 pixels: per chunk it builds A (3
// tiles of 128 (tap, ci) rows x 128 pixels; rows 288..383 stay zero) and B
// (32 co rows x 128 pixels), issues 3 x 8 MMAs into three 32-column
// accumulators and waits for them before the next chunk.  The accumulators
// and the bias gradient are written as this CTA's partial sums; a second
// kernel adds the partials of all CTAs in CTA order, so that the gradient
// (and with it training) does not depend on the order the CTAs finish in.
constexpr int kWgA = 128 * 128 * 2;     // one A tile: 32 KiB
constexpr int kWgB = 32 * 128 * 2;      // 8 KiB
constexpr int kWgSmem = 3 * kWgA + kWgB + 16;
constexpr int kWgMaxCtas = 304;         // about two CTAs per SM
constexpr int kWgPart = kBnK * 32 + 32; // one CTA's partial: dw [co][tap][ci], then db [co]
// partial sums of one sgmf_bn_wgrad call (calls must not overlap on the GPU)
static __device__ float g_wgrad_part[kWgMaxCtas * kWgPart];

struct BnWgradArgs {
  int n, h, w, chunks;
  const uint16_t *x, *dy;   // bf16 [n][h][w][32]
  float *part;              // f32 [gridDim.x][kWgPart] partial sums
  int *err;
};

__global__ void __launch_bounds__(128) k_bn_wgrad(const __grid_constant__ BnWgradArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t *As = sm;
  uint8_t *Bs = sm + 3 * kWgA;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 3 * kWgA + kWgB);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + 3 * kWgA + kWgB + 8);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(slot, 128);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  // the padding rows 288..383 of the third A tile stay zero
  for (int i = tid; i < kWgA / 16; i += 128) reinterpret_cast<uint4 *>(As + 2 * kWgA)[i] = make_uint4(0, 0, 0, 0);
  float dbp[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) dbp[c] = 0.0f;
  const long long P = (long long)a.n * a.h * a.w;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  bool ok = true;
  int issued = 0;
  for (int ch = 0; ch < a.chunks && ok; ++ch) {
    const long long p = ((long long)blockIdx.x * a.chunks + ch) * 128 + tid;
    if ((long long)blockIdx.x * a.chunks * 128 + (long long)ch * 128 >= P) break;   // CTA-uniform
    const bool live = p < P;
    int img = 0, py = 0, px = 0;
    if (live) {
      img = (int)(p / ((long long)a.h * a.w));
      const int r = (int)(p % ((long long)a.h * a.w));
      py = r / a.w;
      px = r % a.w;
    }
    // B: dY of this pixel (column tid), and the bias-gradient partial sums
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.dy + (live ? p : 0) * kBnC);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 v = live ? src[j] : make_uint4(0, 0, 0, 0);
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c0 = 8 * j + 2 * q;
          *reinterpret_cast<uint16_t *>(Bs + cm_off(c0, tid, 16)) = (uint16_t)(u[q] & 0xffffu);
          *reinterpret_cast<uint16_t *>(Bs + cm_off(c0 + 1, tid, 16)) = (uint16_t)(u[q] >> 16);
          dbp[c0] += bf2f((uint16_t)(u[q] & 0xffffu));
          dbp[c0 + 1] += bf2f((uint16_t)(u[q] >> 16));
        }
      }
    }
    // A: X at the 9 taps of this pixel (column tid), rows (tap, ci)
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
      const bool in = live && yy >= 0 && yy < a.h && xx >= 0 && xx < a.w;
      const long long q = in ? ((long long)img * a.h + yy) * a.w + xx : 0;
      const uint4 *src = reinterpret_cast<const uint4 *>(a.x + q * kBnC);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint4 v = in ? src[j] : make_uint4(0, 0, 0, 0);
        const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int m0 = tap * kBnC + 8 * j + 2 * q;
          uint8_t *t0 = As + (m0 >> 7) * kWgA, *t1 = As + ((m0 + 1) >> 7) * kWgA;
          *reinterpret_cast<uint16_t *>(t0 + cm_off(m0 & 127, tid, 16)) = (uint16_t)(u[q] & 0xffffu);
          *reinterpret_cast<uint16_t *>(t1 + cm_off((m0 + 1) & 127, tid, 16)) = (uint16_t)(u[q] >> 16);
        }
      }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t idesc = idesc_bf16(128, 32);
      const uint32_t b0 = smem_u32(Bs);
#pragma unroll 1
      for (int t = 0; t < 3; ++t) {
        const uint32_t a0 = smem_u32(As + t * kWgA);
#pragma unroll 1
        for (int s = 0; s < 8; ++s)
          umma_bf16(tmem + 32 * t, sdesc(a0 + s * 256, 128, 16 * 128), sdesc(b0 + s * 256, 128, 16 * 128), idesc,
                    (ch > 0 || s > 0) ? 1u : 0u);
      }
      umma_commit(bar);
    }
    __syncwarp();
    const bool w_ok = mbar_wait_bounded(bar, (uint32_t)(issued & 1), kWaitLimit);
    ++issued;
    if (!__syncthreads_and(w_ok)) {
      if (tid == 0) set_error(a.err, kErrTimeout);
      mbar_wait_bounded(bar, (uint32_t)((issued - 1) & 1), kWaitLimit);
      ok = false;
    }
    tc_fence_after();
  }
  float *part = a.part + (size_t)blockIdx.x * kWgPart;
#pragma unroll 1
  for (int t = 0; t < 3; ++t) {
    float v[32];
    if (ok && issued > 0) {
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32 * t, v);
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = 0.0f;
    }
    const int m = 128 * t + warp * 32 + lane;   // (tap, ci) row
    if (m < kBnK) {
#pragma unroll
      for (int c = 0; c < 32; ++c) part[c * kBnK + m] = v[c];
    }
  }
  // bias gradient: each warp's sums, then the four warps in order
  __shared__ float dbw[4][32];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    float s = dbp[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dbw[warp][c] = s;
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32)
    part[kBnK * 32 + threadIdx.x] = ((dbw[0][threadIdx.x] + dbw[1][threadIdx.x]) + dbw[2][threadIdx.x]) + dbw[3][threadIdx.x];
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// ---- quarter-resolution input ----------------------------------------------------------
// x[n][y4][x4][c]: c0 = mean(left over the 4 x 4 block) / 255 - 0.5, c1 = mean
// of the valid d-hat in the block / D (0 without one), c2 = valid d-hat / 16;
// channels 3..31 are zero.  Blocks are clipped at the image border.
__global__ void k_bn_input(int n, int W, int H, int D, const uint8_t *__restrict__ left,
                           const int16_t *__restrict__ dhat, uint16_t *__restrict__ x) {
  const int H4 = (H + 3) / 4, W4 = (W + 3) / 4;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * H4 * W4) return;
  const int f = (int)(i / ((long long)H4 * W4));
  const int r = (int)(i % ((long long)H4 * W4));
  const int qy = r / W4, qx = r % W4;
  int sl = 0, cnt = 0, np = 0, sd = 0;
  for (int dy = 0; dy < 4; ++dy)
    for (int dx = 0; dx < 4; ++dx) {
      const int y = 4 * qy + dy, xx = 4 * qx + dx;
      if (y >= H || xx >= W) continue;
      const size_t p = ((size_t)f * H + y) * W + xx;
      sl += left[p];
      ++np;
      const int d = dhat[p];
      if (d >= 0) {
        sd += d;
        ++cnt;
      }
    }
  float v[3];
  v[0] = (float)sl / (255.0f * np) - 0.5f;
  v[1] = cnt ? (float)sd / ((float)cnt * D) : 0.0f;
  v[2] = (float)cnt / 16.0f;
  uint4 *o = reinterpret_cast<uint4 *>(x + i * kBnC);
  o[0] = make_uint4((uint32_t)f2bf(v[0]) | ((uint32_t)f2bf(v[1]) << 16), (uint32_t)f2bf(v[2]), 0, 0);
  o[1] = make_uint4(0, 0, 0, 0);
  o[2] = make_uint4(0, 0, 0, 0);
  o[3] = make_uint4(0, 0, 0, 0);
}

// ---- labels and loss ----------------------------------------------------------------
// labels: per quarter pixel the min / max of the valid disparities of the
// plain output in its 4 x 4 block (lohi[2 i] = lo, [2 i + 1] = hi; -1 without
// one); count += labelled pixels.
__global__ void k_bn_labels(int n, int W, int H, const int16_t *__restrict__ disp, int16_t *__restrict__ lohi,
                            int *count) {
  const int H4 = (H + 3) / 4, W4 = (W + 3) / 4;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * H4 * W4) return;
  const int f = (int)(i / ((long long)H4 * W4));
  const int r = (int)(i % ((long long)H4 * W4));
  const int qy = r / W4, qx = r % W4;
  int lo = 0x7fff, hi = -1;
  for (int dy = 0; dy < 4; ++dy)
    for (int dx = 0; dx < 4; ++dx) {
      const int y = 4 * qy + dy, xx = 4 * qx + dx;
      if (y >= H || xx >= W) continue;
      const int d = disp[((size_t)f * H + y) * W + xx];
      if (d >= 0) {
        lo = min(lo, d);
        hi = max(hi, d);
      }
    }
  lohi[2 * i] = (int16_t)(hi >= 0 ? lo : -1);
  lohi[2 * i + 1] = (int16_t)hi;
  if (hi >= 0) atomicAdd(count, 1);
}

// loss and its gradient with respect to the last layer's outputs (channels
// 0..2; the rest get 0): see the band loss definition in the header.
__global__ void k_bn_loss(long long npix, int D, const float *__restrict__ out, const int16_t *__restrict__ lohi,
                          const int *__restrict__ count, uint16_t *__restrict__ grad, float *loss, float lam_c,
                          float lam_w) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < npix;   // no early return: the warp reduction below needs every lane
  const float inv = 1.0f / (float)max(*count, 1);
  const long long ii = live ? i : 0;
  const float o0 = out[ii * kBnC], o1 = out[ii * kBnC + 1], o2 = out[ii * kBnC + 2];
  const int lo = lohi[2 * ii], hi = live ? lohi[2 * ii + 1] : -1;
  float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, l = 0.0f;
  if (hi >= 0) {
    const float c = D * o0;
    const float s1 = 1.0f / (1.0f + expf(-o1));
    const float w = 8.0f + 40.0f * s1;
    const float q = 1.0f / (1.0f + expf(-o2));
    const float ct = 0.5f * (lo + hi);
    const float wt = fminf(fmaxf(0.5f * (hi - lo) + 2.0f, 8.0f), 48.0f);
    const float y = (c - w <= (float)lo && (float)hi <= c + w) ? 1.0f : 0.0f;
    const float sc = c > ct ? 1.0f : (c < ct ? -1.0f : 0.0f);
    const float sw = w > wt ? 1.0f : (w < wt ? -1.0f : 0.0f);
    g0 = lam_c * sc * inv;
    g1 = lam_w * sw / D * 40.0f * s1 * (1.0f - s1) * inv;
    g2 = (q - y) * inv;
    l = lam_c * fabsf(c - ct) / D + lam_w * fabsf(w - wt) / D -
        (y * logf(q + 1e-12f) + (1.0f - y) * logf(1.0f - q + 1e-12f));
  }
  if (live) {
    uint4 *o = reinterpret_cast<uint4 *>(grad + i * kBnC);
    o[0] = make_uint4((uint32_t)f2bf(g0) | ((uint32_t)f2bf(g1) << 16), (uint32_t)f2bf(g2), 0, 0);
    o[1] = make_uint4(0, 0, 0, 0);
    o[2] = make_uint4(0, 0, 0, 0);
    o[3] = make_uint4(0, 0, 0, 0);
  }
  float s = l * inv;
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0 && s != 0.0f) atomicAdd(loss, s);
}

// ---- Adam (fp32 master weights, bf16 copy) ---------------------------------------------
__global__ void k_bn_adam(int count, float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                          const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2,
                          uint16_t *__restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) wb[i] = f2bf(wi);
}

// ---- training batches and weight copies ----------------------------------------------------
// dst row i = src row idx[i] (rows of row_vec elements of type T, 16 or 4
// bytes): a training batch gathered from the resident training set; an
// index outside [0, rows) leaves its destination row untouched
template <typename T>
__global__ void __launch_bounds__(256) k_bn_gather(int n, const int *__restrict__ idx, long long rows, long long row_vec,
                                                   const T *__restrict__ src, T *__restrict__ dst) {
  const int i = blockIdx.y;
  const int r = idx[i];
  if (r < 0 || (long long)r >= rows) return;
  const T *s = src + (long long)r * row_vec;
  T *d = dst + (long long)i * row_vec;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < row_vec; j += (long long)gridDim.x * blockDim.x)
    d[j] = s[j];
}

// bf16 copy (round to nearest, ties to even) of count f32 values
__global__ void __launch_bounds__(256) k_bn_to_bf16(int count, const float *__restrict__ w, uint16_t *__restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) wb[i] = f2bf(w[i]);
}

// ---- network output -> band starts per tile ----------------------------------------------
// For each tile (kBandTile / 4 quarter pixels a side): the union [lo_u, hi_u] of the pixels'
// bands [c - w, c + w]; band start lo = round((lo_u + hi_u) / 2) - B / 2,
// clamped to [0, D - B].  A tile is uncertain when the smallest confidence in
// it is below conf_min or the union is wider than B; uncertain[f] counts the
// uncertain tiles of frame f.
__global__ void k_bn_tiles(int n, int W, int H, int D, int B, float conf_min, const float *__restrict__ out,
                           int16_t *__restrict__ lo_tiles, int *uncertain) {
  constexpr int Q = kBandTile / 4;   // quarter pixels per tile side
  const int H4 = (H + 3) / 4, W4 = (W + 3) / 4, th = (H + kBandTile - 1) / kBandTile,
            tw = (W + kBandTile - 1) / kBandTile;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * th * tw) return;
  const int f = (int)(i / ((long long)th * tw));
  const int r = (int)(i % ((long long)th * tw));
  const int ty = r / tw, tx = r % tw;
  float lo_u = 1e30f, hi_u = -1e30f, qmin = 1.0f;
  for (int dy = 0; dy < Q; ++dy)
    for (int dx = 0; dx < Q; ++dx) {
      const int qy = Q * ty + dy, qx = Q * tx + dx;
      if (qy >= H4 || qx >= W4) continue;
      const float *o = out + (((long long)f * H4 + qy) * W4 + qx) * kBnC;
      const float c = D * o[0];
      const float w = 8.0f + 40.0f / (1.0f + expf(-o[1]));
      const float q = 1.0f / (1.0f + expf(-o[2]));
      lo_u = fminf(lo_u, c - w);
      hi_u = fmaxf(hi_u, c + w);
      qmin = fminf(qmin, q);
    }
  const int mid = __float2int_rn(0.5f * (lo_u + hi_u));
  lo_tiles[i] = (int16_t)min(max(mid - B / 2, 0), D - B);
  if (qmin < conf_min || hi_u - lo_u > (float)B) atomicAdd(uncertain + f, 1);
}

// per frame: gate[f] = value when frame f has at most max_tiles uncertain
// tiles, else `otherwise` (or the gate word is kept when otherwise < 0)
__global__ void k_bn_decide(int n, int max_tiles, const int *__restrict__ uncertain, int value, int otherwise,
                            int *__restrict__ gate) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  if (uncertain[f] <= max_tiles)
    gate[f] = value;
  else if (otherwise >= 0)
    gate[f] = otherwise;
}

}  // namespace sgmf

using namespace sgmf;

static sgmf_status bn_launch(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return SGMF_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  set_noctx_error(buf);
  return SGMF_ERR_CUDA;
}

extern "C" sgmf_status sgmf_bn_pack(const uint16_t *w, uint16_t *packed_fwd, uint16_t *packed_dgrad, void *stream) {
  if (!w) return SGMF_ERR_ARG;
  k_bn_pack<<<(kBnC * kBnK + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(w, packed_fwd, packed_dgrad);
  return bn_launch(cudaGetLastError(), "sgmf_bn_pack");
}

extern "C" sgmf_status sgmf_bn_conv(int n, int h, int w, const uint16_t *x, const uint16_t *packed, const float *bias,
                                    int relu, const uint16_t *mask, uint16_t *y, float *yf, int *err, void *stream) {
  if (n < 1 || h < 1 || w < 1 || !x || !packed || !err || (!y && !yf)) return SGMF_ERR_ARG;
  const long long ntile = (long long)n * h * ((w + kCvM - 1) / kCvM);
  // one wave of about four CTAs per SM, each walking consecutive tiles with
  // its weights staged once
  int sms = 0;
  const cudaError_t e = sm_count(&sms);
  if (e != cudaSuccess) return bn_launch(e, "sgmf_bn_conv");
  const long long slots = 4LL * std::max(sms, 1);
  const int tiles = (int)std::max<long long>(1, std::min<long long>(32, (ntile + slots - 1) / slots));
  BnConvArgs a{n, h, w, x, reinterpret_cast<const uint4 *>(packed), bias, relu, mask, y, yf, err};
  k_bn_conv<<<(unsigned)((ntile + tiles - 1) / tiles), 128, kCvSmem, static_cast<cudaStream_t>(stream)>>>(a, tiles);
  return bn_launch(cudaGetLastError(), "sgmf_bn_conv");
}

// dw / db += the partials of `ctas` CTAs, added in CTA order
__global__ void __launch_bounds__(256) k_bn_wgrad_sum(const float *__restrict__ part, int ctas, float *dw, float *db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= kWgPart) return;
  float s = 0.0f;
  for (int b = 0; b < ctas; ++b) s += part[(size_t)b * kWgPart + o];
  if (o < kBnK * 32)
    dw[o] += s;
  else
    db[o - kBnK * 32] += s;
}

extern "C" sgmf_status sgmf_bn_wgrad(int n, int h, int w, const uint16_t *x, const uint16_t *dy, float *dw, float *db,
                                     int *err, void *stream) {
  if (n < 1 || h < 1 || w < 1 || !x || !dy || !dw || !db || !err) return SGMF_ERR_ARG;
  static bool attr[64] = {};
  const cudaError_t ea = once_per_device(attr, [](int) {
    return cudaFuncSetAttribute(k_bn_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
  });
  if (ea != cudaSuccess) return bn_launch(ea, "sgmf_bn_wgrad attribute");
  const long long P = (long long)n * h * w;
  const long long nchunk = (P + 127) / 128;
  const int chunks = (int)((nchunk + kWgMaxCtas - 1) / kWgMaxCtas);
  const unsigned grid = (unsigned)((nchunk + chunks - 1) / chunks);   // <= kWgMaxCtas
  float *part = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&part), g_wgrad_part);
  if (e != cudaSuccess) return bn_launch(e, "sgmf_bn_wgrad scratch");
  BnWgradArgs a{n, h, w, chunks, x, dy, part, err};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_bn_wgrad<<<grid, 128, kWgSmem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bn_launch(e, "sgmf_bn_wgrad");
  k_bn_wgrad_sum<<<(kWgPart + 255) / 256, 256, 0, s>>>(part, (int)grid, dw, db);
  return bn_launch(cudaGetLastError(), "sgmf_bn_wgrad");
}

extern "C" sgmf_status sgmf_bn_input(int n, int width, int height, int max_disp, const uint8_t *left,
                                     const int16_t *dhat, uint16_t *x, void *stream) {
  if (n < 1 || width < 1 || height < 1 || !left || !dhat || !x) return SGMF_ERR_ARG;
  const long long N4 = (long long)n * ((height + 3) / 4) * ((width + 3) / 4);
  k_bn_input<<<(unsigned)((N4 + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, width, height, max_disp,
                                                                                         left, dhat, x);
  return bn_launch(cudaGetLastError(), "sgmf_bn_input");
}

extern "C" sgmf_status sgmf_bn_labels(int n, int width, int height, const int16_t *disp, int16_t *lohi, int *count,
                                      void *stream) {
  if (n < 1 || width < 1 || height < 1 || !disp || !lohi || !count) return SGMF_ERR_ARG;
  const long long N4 = (long long)n * ((height + 3) / 4) * ((width + 3) / 4);
  k_bn_labels<<<(unsigned)((N4 + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, width, height, disp,
                                                                                          lohi, count);
  return bn_launch(cudaGetLastError(), "sgmf_bn_labels");
}

extern "C" sgmf_status sgmf_bn_loss(long long npix, int max_disp, const float *out, const int16_t *lohi,
                                    const int *count, uint16_t *grad, float *loss, float lam_c, float lam_w,
                                    void *stream) {
  if (npix < 1 || !out || !lohi || !count || !grad || !loss) return SGMF_ERR_ARG;
  k_bn_loss<<<(unsigned)((npix + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      npix, max_disp, out, lohi, count, grad, loss, lam_c, lam_w);
  return bn_launch(cudaGetLastError(), "sgmf_bn_loss");
}

extern "C" sgmf_status sgmf_bn_adam(int count, float *w, float *m, float *v, const float *g, float lr, float b1,
                                    float b2, float eps, int step, uint16_t *w_bf16, void *stream) {
  if (count < 1 || !w || !m || !v || !g || step < 1) return SGMF_ERR_ARG;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_bn_adam<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(count, w, m, v, g, lr, b1, b2, eps,
                                                                                 c1, c2, w_bf16);
  return bn_launch(cudaGetLastError(), "sgmf_bn_adam");
}

extern "C" sgmf_status sgmf_bn_tiles(int n, int width, int height, int max_disp, int band, float conf_min,
                                     const float *out, int16_t *lo_tiles, int *uncertain, void *stream) {
  if (n < 1 || width < 1 || height < 1 || band < 1 || band > max_disp || !out || !lo_tiles || !uncertain)
    return SGMF_ERR_ARG;
  const long long NT = (long long)n * ((height + kBandTile - 1) / kBandTile) * ((width + kBandTile - 1) / kBandTile);
  k_bn_tiles<<<(unsigned)((NT + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, width, height, max_disp, band, conf_min, out, lo_tiles, uncertain);
  return bn_launch(cudaGetLastError(), "sgmf_bn_tiles");
}

extern "C" sgmf_status sgmf_bn_decide(int n, int tiles, float max_frac, const int *uncertain, int value,
                                      int otherwise, int *gate, void *stream) {
  if (n < 1 || tiles < 1 || !(max_frac >= 0.0f) || !uncertain || !gate) return SGMF_ERR_ARG;
  const int max_tiles = (int)std::min<double>((double)max_frac * tiles, (double)tiles);
  k_bn_decide<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, max_tiles, uncertain, value,
                                                                                 otherwise, gate);
  return bn_launch(cudaGetLastError(), "sgmf_bn_decide");
}

extern "C" sgmf_status sgmf_bn_gather(int n, const int *idx, long long rows, long long row_bytes, const void *src,
                                      void *dst, void *stream) {
  if (n < 1 || n > 65535 || rows < 1 || row_bytes < 4 || row_bytes % 4 != 0 || !idx || !src || !dst ||
      reinterpret_cast<uintptr_t>(src) % 4 != 0 || reinterpret_cast<uintptr_t>(dst) % 4 != 0)
    return SGMF_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // 16-byte elements when every row starts on a 16-byte boundary, else words
  const bool v16 = row_bytes % 16 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(dst) % 16 == 0;
  const long long vec = row_bytes / (v16 ? 16 : 4);
  const unsigned bx = (unsigned)std::min<long long>((vec + 255) / 256, 64);
  if (v16)
    k_bn_gather<uint4><<<dim3(bx, (unsigned)n), 256, 0, s>>>(n, idx, rows, vec, static_cast<const uint4 *>(src),
                                                             static_cast<uint4 *>(dst));
  else
    k_bn_gather<uint32_t><<<dim3(bx, (unsigned)n), 256, 0, s>>>(n, idx, rows, vec, static_cast<const uint32_t *>(src),
                                                                static_cast<uint32_t *>(dst));
  return bn_launch(cudaGetLastError(), "sgmf_bn_gather");
}

extern "C" sgmf_status sgmf_bn_to_bf16(int count, const float *w, uint16_t *w_bf16, void *stream) {
  if (count < 1 || !w || !w_bf16) return SGMF_ERR_ARG;
  k_bn_to_bf16<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(count, w, w_bf16);
  return bn_launch(cudaGetLastError(), "sgmf_bn_to_bf16");
}
