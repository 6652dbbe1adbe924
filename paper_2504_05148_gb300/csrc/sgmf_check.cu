// sgmf_check.cu -- three-view stereo-LiDAR consistency check, Eq. 6 (Sec. IV-C).
#include <cstdint>

#include "sgmf_internal.cuh"

namespace sgmf {

// D^{c*}_p = d*_p when
//   the stereo term holds: q_m = (x - d*, y) is in the image and
//   |d*_p - d'(q_m)| <= lr, or
//   the LiDAR term holds: some valid raw d-bar_q, q in the (2rc+1)^2 window
//   K_p (clipped), has |d*_p - d-bar_q| <= tc -- i.e. the window's presence
//   masks have a bit in [d* - tc, d* + tc];
// otherwise -1.  The raw map d-bar is used, never d-hat.  `consistency`
// selects the Table V variants.  With the sub-pixel fit on, a kept pixel
// carries its sub-pixel disparity (1/16 px) instead of d*; the test itself
// is always on the integer d*.
//
// boxC holds the row ORs of the presence masks (|x' - x| <= rc); the LiDAR
// term ORs the 2 rc + 1 rows of the window at the pixel itself, and only
// where the result decides the output (in the default mode, where the
// stereo term fails: a small fraction of the pixels).
__global__ void __launch_bounds__(256) k_consistency(KParams k, Buffers b0, int16_t *__restrict__ out) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= k.W || y >= k.H) return;
  const Buffers b = frame_view(k, b0, blockIdx.z);
  if (gated_off(b.gate, k.gate_run)) return;
  out += (size_t)blockIdx.z * frame_px(k);
  const size_t p = (size_t)y * k.W + x;
  const int ds = b.dstar[p];
  bool stereo_ok = false, lidar_ok = false;
  if (k.consistency != 2 && k.consistency != 3) {
    const int xm = x - ds;
    // (d' is always valid for the plain method; the banded mode marks a right
    // pixel whose diagonal meets no band with -1, and the term then fails)
    const int dp = xm >= 0 ? (int)b.dprime[(size_t)y * k.W + xm] : -1;
    stereo_ok = dp >= 0 && abs(ds - dp) <= k.lr;
  }
  if (k.consistency == 2 || (k.consistency == 0 && !stereo_ok)) {
    const int lo = max(ds - k.tc, 0), hi = min(ds + k.tc, k.D - 1);
    const size_t plane = (size_t)k.W * k.H;
    const int y0 = max(y - k.rc, 0), y1 = min(y + k.rc, k.H - 1);
    for (int w = lo >> 5; w <= (hi >> 5) && !lidar_ok; ++w) {
      const int a = max(lo - 32 * w, 0), e = min(hi - 32 * w, 31);   // bit range [a, e] of word w
      const uint32_t upto = e == 31 ? 0xffffffffu : ((1u << (e + 1)) - 1u);
      const uint32_t rng = upto & ~((1u << a) - 1u);
      const uint32_t *col = b.boxC + w * plane + x;
      // the window's rows, eight loads in flight at a time
      for (int yy = y0; yy <= y1 && !lidar_ok; yy += 8) {
        uint32_t acc = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (yy + j <= y1) acc |= col[(size_t)(yy + j) * k.W];
        lidar_ok = (acc & rng) != 0u;
      }
    }
  }
  bool ok;
  switch (k.consistency) {
    case 1: ok = stereo_ok; break;
    case 2: ok = lidar_ok; break;
    case 3: ok = true; break;
    default: ok = stereo_ok || lidar_ok; break;
  }
  const int16_t v = k.subpixel ? b.dsub[p] : (int16_t)ds;
  out[p] = ok ? v : (int16_t)-1;
}

cudaError_t launch_consistency(const KParams &k, const Buffers &b, int nf, int16_t *out, cudaStream_t s) {
  dim3 grid((k.W + 31) / 32, (k.H + 7) / 8, nf);
  k_consistency<<<grid, 256, 0, s>>>(k, b, out);
  return cudaGetLastError();
}

}  // namespace sgmf
