/*
 * sgmf_oracle.c -- plain, slow, single-threaded CPU statement of the
 * stereo-LiDAR SGM pipeline of "Stereo-LiDAR Fusion by Semi-Global Matching
 * with Discrete Disparity-Matching Cost and Semidensification" (Yao,
 * Ishikawa, Oishi, RA-L 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no source, header, table or helper
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Every stage is written as the literal definition: loops over pixels p,
 * disparities d and path directions r, int32 arithmetic, no SIMD, no fusion,
 * no blocking.  Each function names the passage of the paper it follows.
 * Where the paper is silent the function states the reading it takes.
 *
 * Conventions shared with the callers (documented, not code):
 *   images are row-major H x W, index y*W + x;
 *   volumes are row-major H x W x D, index (y*W + x)*D + d;
 *   an invalid disparity is -1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SGMFO_INVALID (-1)

/* consistency modes (Table V of the paper: stereo, camera-LiDAR, stereo-LiDAR) */
#define SGMFO_CHECK_STEREO_LIDAR 0
#define SGMFO_CHECK_STEREO 1
#define SGMFO_CHECK_LIDAR 2
#define SGMFO_CHECK_NONE 3

/* census kinds */
#define SGMFO_CENSUS_CS9X7 0   /* centre-symmetric 9x7: 31 bits */
#define SGMFO_CENSUS_9X7 1     /* full 9x7 against the centre: 62 bits */

typedef struct {
    int32_t p1, p2;              /* SGM penalties, Eq. 1/2, Table II: 10, 120 */
    int32_t q1, q2;              /* DDC penalties, Eq. 4, Table II: 5, 160 */
    int32_t alpha_num, alpha_den;/* alpha = num/den, Eq. 4, Table II: 0.7 */
    int32_t ts, rs;              /* semidensification, Eq. 5, Table II: 2, 6 */
    int32_t tc, rc;              /* consistency, Eq. 6, Table II: 2, 20 */
    int32_t lr_max_diff;         /* stereo term of Eq. 6: |d* - d'| <= 1 */
    int32_t census;              /* SGMFO_CENSUS_* */
    int32_t semidense;           /* 1 = SDSGM, 0 = DSGM (Table I) */
    int32_t consistency;         /* SGMFO_CHECK_* */
    int32_t num_paths;           /* 8 (Sec. III) or 4 */
    int32_t subpixel;            /* 1: output in 1/16 px after the parabola fit (Sec. III) */
} sgmfo_params;

static int iabs_(int v) { return v < 0 ? -v : v; }

/* ------------------------------------------------------------------------ */
/* Sparse disparity map D-bar (Sec. IV, first paragraph).  The paper takes
 * d-bar in N u {invalid}; the input here is a float map with 0 meaning "no
 * return".  Reading: d-bar = rint(f) (IEEE round-half-to-even in the default
 * rounding mode) when f is finite, f > 0 and rint(f) <= D-1; otherwise
 * invalid.  lidar == NULL means no LiDAR at all. */
void sgmfo_lidar(int W, int H, int D, const float *lidar, int16_t *dbar)
{
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int v = SGMFO_INVALID;
            if (lidar != NULL) {
                float f = lidar[(size_t)y * W + x];
                if (isfinite(f) && f > 0.0f) {
                    float r = rintf(f);
                    if (r <= (float)(D - 1)) v = (int)r;
                }
            }
            dbar[(size_t)y * W + x] = (int16_t)v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Census transform (Sec. IV-A: the stereo cost is the Hamming distance of
 * census-transformed images, after Spangenberg et al.).  The paper gives no
 * window; reading: 9 wide x 7 high.
 *
 * Offsets o = (dx, dy), dx in [-4, 4], dy in [-3, 3], are enumerated in
 * raster order (dy outer, dx inner) with the centre left out; the k-th
 * enumerated offset sets bit k.
 *   SGMFO_CENSUS_9X7:  all 62 offsets; bit = I(p+o) > I(p).
 *   SGMFO_CENSUS_CS9X7: the 31 offsets before the centre in raster order;
 *                       bit = I(p+o) > I(p-o)  (centre-symmetric pairs).
 * A bit whose compared samples are not all inside the image is 0. */
void sgmfo_census(int W, int H, const uint8_t *img, int kind, uint64_t *out)
{
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            uint64_t c = 0;
            int k = 0;
            for (int dy = -3; dy <= 3; ++dy) {
                for (int dx = -4; dx <= 4; ++dx) {
                    if (dx == 0 && dy == 0) {
                        if (kind == SGMFO_CENSUS_CS9X7) goto done; /* half window */
                        continue;
                    }
                    int xa = x + dx, ya = y + dy;
                    int bit = 0;
                    if (kind == SGMFO_CENSUS_CS9X7) {
                        int xb = x - dx, yb = y - dy;
                        if (xa >= 0 && xa < W && ya >= 0 && ya < H &&
                            xb >= 0 && xb < W && yb >= 0 && yb < H)
                            bit = img[(size_t)ya * W + xa] > img[(size_t)yb * W + xb];
                    } else {
                        if (xa >= 0 && xa < W && ya >= 0 && ya < H)
                            bit = img[(size_t)ya * W + xa] > img[(size_t)y * W + x];
                    }
                    if (bit) c |= (uint64_t)1 << k;
                    ++k;
                }
            }
        done:
            out[(size_t)y * W + x] = c;
        }
    }
}

int sgmfo_census_bits(int kind) { return kind == SGMFO_CENSUS_CS9X7 ? 31 : 62; }

/* ------------------------------------------------------------------------ */
/* Hamming matching cost H(p, d) (Sec. IV-A): the number of differing census
 * bits between the left pixel (x, y) and the right pixel (x - d, y).
 * Reading: where x - d < 0 the right pixel does not exist and H is the
 * number of census bits (the largest possible distance). */
void sgmfo_hamming(int W, int H, int D, const uint64_t *cl, const uint64_t *cr,
                   int nbits, int32_t *hv)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int d = 0; d < D; ++d) {
                int h = nbits;
                if (x - d >= 0)
                    h = __builtin_popcountll(cl[(size_t)y * W + x] ^ cr[(size_t)y * W + x - d]);
                hv[((size_t)y * W + x) * D + d] = h;
            }
}

/* ------------------------------------------------------------------------ */
/* Semidensification, Eq. 5 (Sec. IV-B).  For every pixel p, the candidates
 * are the valid sparse disparities d-bar_q of the pixels q in the
 * (2 rs + 1) x (2 rs + 1) window M_p centred on p (clipped to the image,
 * p included).  d-hat_p is the candidate with the smallest H(p, d-bar_q)
 * when that smallest cost is below ts; otherwise d-hat_p = d-bar_p, which
 * may be invalid.  Ties in H (which the paper does not order) go to the
 * smaller disparity. */
void sgmfo_semidense(int W, int H, int D, const int16_t *dbar, const int32_t *hv,
                     int ts, int rs, int16_t *dhat)
{
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int best_h = 0x7fffffff, best_d = SGMFO_INVALID;
            for (int qy = y - rs; qy <= y + rs; ++qy) {
                if (qy < 0 || qy >= H) continue;
                for (int qx = x - rs; qx <= x + rs; ++qx) {
                    if (qx < 0 || qx >= W) continue;
                    int dq = dbar[(size_t)qy * W + qx];
                    if (dq < 0) continue;
                    int h = hv[((size_t)y * W + x) * D + dq];
                    if (h < best_h || (h == best_h && dq < best_d)) {
                        best_h = h;
                        best_d = dq;
                    }
                }
            }
            if (best_d >= 0 && best_h < ts)
                dhat[(size_t)y * W + x] = (int16_t)best_d;
            else
                dhat[(size_t)y * W + x] = dbar[(size_t)y * W + x];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Joint cost C-bar with the Discrete Disparity-matching Cost, Eq. 4
 * (Sec. IV-A), using the prior map `prior` (d-hat for SDSGM, d-bar for DSGM).
 *   C-bar = (1 - alpha) H + alpha * q,
 *   q = 0 if d = prior, q1 if |d - prior| = 1, q2 if |d - prior| > 1.
 * Readings:
 *   - where the prior is invalid the DDC is not applied (Sec. IV-B: DDC acts
 *     only where a sparse value exists) and C-bar = H;
 *   - costs are integers: with alpha = a/b,
 *       C-bar = floor(((b - a) H + a q + floor(b/2)) / b),
 *     the real value of Eq. 4 rounded half up. */
void sgmfo_ddc(int W, int H, int D, const int32_t *hv, const int16_t *prior,
               int q1, int q2, int a, int b, int32_t *cv)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int pd = prior[(size_t)y * W + x];
            for (int d = 0; d < D; ++d) {
                size_t i = ((size_t)y * W + x) * D + d;
                int h = hv[i];
                if (pd < 0) {
                    cv[i] = h;
                } else {
                    int q;
                    if (d == pd) q = 0;
                    else if (iabs_(d - pd) == 1) q = q1;
                    else q = q2;
                    cv[i] = ((b - a) * h + a * q + b / 2) / b;
                }
            }
        }
}

/* ------------------------------------------------------------------------ */
/* One SGM path, Eq. 2 (Sec. III).  The path direction is r = (rx, ry):
 * L_r(p, .) is built from L_r(p - r, .).
 *   L_r(p, d) = C(p, d) + min{ L_r(p-r, d),
 *                              L_r(p-r, d-1) + P1,
 *                              L_r(p-r, d+1) + P1,
 *                              min_i L_r(p-r, i) + P2 }
 *               - min_k L_r(p-r, k).
 * Readings: where p - r is outside the image, p starts the path and
 * L_r(p, d) = C(p, d); the d-1 and d+1 terms are left out where that
 * disparity is outside [0, D-1].
 * Pixels are visited in raster order of the quadrant that has p - r
 * before p. */
void sgmfo_path(int W, int H, int D, const int32_t *cv, int p1, int p2,
                int rx, int ry, int32_t *lv)
{
    for (int iy = 0; iy < H; ++iy) {
        int y = ry >= 0 ? iy : H - 1 - iy;
        for (int ix = 0; ix < W; ++ix) {
            int x = rx >= 0 ? ix : W - 1 - ix;
            int px = x - rx, py = y - ry;
            size_t o = ((size_t)y * W + x) * D;
            if (px < 0 || px >= W || py < 0 || py >= H) {
                for (int d = 0; d < D; ++d) lv[o + d] = cv[o + d];
                continue;
            }
            size_t po = ((size_t)py * W + px) * D;
            int m = 0x7fffffff;
            for (int k = 0; k < D; ++k)
                if (lv[po + k] < m) m = lv[po + k];
            for (int d = 0; d < D; ++d) {
                int best = lv[po + d];
                if (d - 1 >= 0 && lv[po + d - 1] + p1 < best) best = lv[po + d - 1] + p1;
                if (d + 1 < D && lv[po + d + 1] + p1 < best) best = lv[po + d + 1] + p1;
                if (m + p2 < best) best = m + p2;
                lv[o + d] = cv[o + d] + best - m;
            }
        }
    }
}

/* The path directions of Sec. III: horizontal, vertical and diagonal, eight
 * in all; the first four (horizontal and vertical) when num_paths == 4. */
static const int kDirs[8][2] = {
    {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};

int sgmfo_direction(int i, int *rx, int *ry)
{
    if (i < 0 || i >= 8) return -1;
    *rx = kDirs[i][0];
    *ry = kDirs[i][1];
    return 0;
}

/* Aggregate cost S(p, d) = sum_r L_r(p, d), the quantity minimised in Eq. 3.
 * Returns 0, or -1 if the scratch volume could not be allocated. */
int sgmfo_aggregate(int W, int H, int D, const int32_t *cv, int p1, int p2,
                    int num_paths, int32_t *sv)
{
    size_t n = (size_t)W * H * D;
    int32_t *lv = (int32_t *)malloc(n * sizeof(int32_t));
    if (lv == NULL) return -1;
    memset(sv, 0, n * sizeof(int32_t));
    for (int i = 0; i < num_paths; ++i) {
        sgmfo_path(W, H, D, cv, p1, p2, kDirs[i][0], kDirs[i][1], lv);
        for (size_t j = 0; j < n; ++j) sv[j] += lv[j];
    }
    free(lv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Winner-takes-all, Eq. 3: d*_p = argmin_d S(p, d).
 * The disparity of the matching pixel in the other view (Sec. IV-C, the d'
 * of Eq. 6) is read, as in Hirschmuller's SGM, off the same aggregate along
 * the epipolar diagonal: d'(x', y) = argmin over d with x' + d < W of
 * S(x' + d, y, d).  Ties go to the smaller disparity in both. */
void sgmfo_wta(int W, int H, int D, const int32_t *sv, int16_t *dstar, int16_t *dprime)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int32_t *s = sv + ((size_t)y * W + x) * D;
            int bd = 0;
            for (int d = 1; d < D; ++d)
                if (s[d] < s[bd]) bd = d;
            dstar[(size_t)y * W + x] = (int16_t)bd;
        }
    for (int y = 0; y < H; ++y)
        for (int xr = 0; xr < W; ++xr) {
            int bd = SGMFO_INVALID, bs = 0x7fffffff;
            for (int d = 0; d < D && xr + d < W; ++d) {
                int s = sv[((size_t)y * W + xr + d) * D + d];
                if (s < bs) {
                    bs = s;
                    bd = d;
                }
            }
            dprime[(size_t)y * W + xr] = (int16_t)bd;
        }
}

/* ------------------------------------------------------------------------ */
/* Sub-pixel disparity (Sec. III, the step after Eq. 3): the parabola through
 * (d* - 1, S(d* - 1)), (d*, S(d*)), (d* + 1, S(d* + 1)) has its vertex at
 *   d* + (S(d* - 1) - S(d* + 1)) / (2 (S(d* - 1) - 2 S(d*) + S(d* + 1))).
 * Readings: the result is kept in fixed point with 4 fraction bits (1/16 px),
 * the fraction rounded half up; where d* = 0 or d* = D - 1 one neighbour is
 * missing and the result is 16 d*.  d* being the smallest argmin, S(d* - 1)
 * > S(d*) <= S(d* + 1): the denominator is positive and the offset lies in
 * [-1/2, 1/2], i.e. [-8, 8] sixteenths. */
static long floor_div_(long a, long b) /* b > 0 */
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

void sgmfo_subpixel(int W, int H, int D, const int32_t *sv, const int16_t *dstar, int16_t *dsub)
{
    for (size_t p = 0; p < (size_t)W * H; ++p) {
        const int ds = dstar[p];
        if (ds <= 0 || ds >= D - 1) {
            dsub[p] = (int16_t)(16 * ds);
            continue;
        }
        const int32_t *s = sv + p * D;
        const long num = (long)s[ds - 1] - s[ds + 1];
        const long den = 2 * ((long)s[ds - 1] - 2L * s[ds] + s[ds + 1]);
        /* 16 num / den rounded half up = floor((32 num + den) / (2 den)) */
        dsub[p] = (int16_t)(16 * ds + floor_div_(32 * num + den, 2 * den));
    }
}

/* ------------------------------------------------------------------------ */
/* Stereo-LiDAR consistency check, Eq. 6 (Sec. IV-C).  d*_p is kept when
 *   the stereo term holds: the matching pixel q_m = (x - d*, y) exists and
 *   |d*_p - d'(q_m)| <= lr_max_diff (1 in Eq. 6), or
 *   the LiDAR term holds: some valid raw sparse disparity d-bar_q with q in
 *   the (2 rc + 1) x (2 rc + 1) window K_p (clipped to the image) has
 *   |d*_p - d-bar_q| <= tc.
 * The raw map d-bar is used, not d-hat (stated after Eq. 6).  Otherwise the
 * output is invalid (-1).  `mode` selects the ablation variants of Table V. */
static void consistency_(int W, int H, const int16_t *dstar, const int16_t *dprime,
                         const int16_t *dbar, int tc, int rc, int lr_max_diff, int mode,
                         int need_dprime, int16_t *out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int ds = dstar[(size_t)y * W + x];
            int stereo_ok = 0, lidar_ok = 0;
            int xm = x - ds;
            if (xm >= 0 && (!need_dprime || dprime[(size_t)y * W + xm] >= 0) &&
                iabs_(ds - dprime[(size_t)y * W + xm]) <= lr_max_diff)
                stereo_ok = 1;
            for (int qy = y - rc; qy <= y + rc && !lidar_ok; ++qy) {
                if (qy < 0 || qy >= H) continue;
                for (int qx = x - rc; qx <= x + rc; ++qx) {
                    if (qx < 0 || qx >= W) continue;
                    int dq = dbar[(size_t)qy * W + qx];
                    if (dq >= 0 && iabs_(ds - dq) <= tc) {
                        lidar_ok = 1;
                        break;
                    }
                }
            }
            int ok;
            switch (mode) {
            case SGMFO_CHECK_STEREO: ok = stereo_ok; break;
            case SGMFO_CHECK_LIDAR: ok = lidar_ok; break;
            case SGMFO_CHECK_NONE: ok = 1; break;
            default: ok = stereo_ok || lidar_ok; break;
            }
            out[(size_t)y * W + x] = (int16_t)(ok ? ds : SGMFO_INVALID);
        }
}

void sgmfo_consistency(int W, int H, const int16_t *dstar, const int16_t *dprime,
                       const int16_t *dbar, int tc, int rc, int lr_max_diff, int mode,
                       int16_t *out)
{
    consistency_(W, H, dstar, dprime, dbar, tc, rc, lr_max_diff, mode, 0, out);
}

/* ------------------------------------------------------------------------ */
/* The whole pipeline of Fig. 1: semidensification (optional, Table I),
 * SGM with DDC, WTA, three-view check.  With prm->subpixel the pixels that
 * pass the check carry the sub-pixel disparity in 1/16 px instead of d*
 * (invalid stays -1).  Every non-NULL dump pointer receives the
 * corresponding intermediate.  Returns 0, or -1 on allocation failure. */
int sgmfo_compute(const sgmfo_params *prm, int W, int H, int D,
                  const uint8_t *left, const uint8_t *right, const float *lidar,
                  int16_t *out,
                  int16_t *dump_dbar, uint64_t *dump_cl, uint64_t *dump_cr,
                  int16_t *dump_dhat, int32_t *dump_cost, int32_t *dump_sum,
                  int16_t *dump_dstar, int16_t *dump_dprime)
{
    size_t n = (size_t)W * H, nv = n * (size_t)D;
    int16_t *dbar = (int16_t *)malloc(n * sizeof(int16_t));
    int16_t *dhat = (int16_t *)malloc(n * sizeof(int16_t));
    int16_t *dstar = (int16_t *)malloc(n * sizeof(int16_t));
    int16_t *dprime = (int16_t *)malloc(n * sizeof(int16_t));
    uint64_t *cl = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *cr = (uint64_t *)malloc(n * sizeof(uint64_t));
    int32_t *hv = (int32_t *)malloc(nv * sizeof(int32_t));
    int32_t *cv = (int32_t *)malloc(nv * sizeof(int32_t));
    int rc = -1;
    if (!dbar || !dhat || !dstar || !dprime || !cl || !cr || !hv || !cv) goto out;

    sgmfo_lidar(W, H, D, lidar, dbar);
    sgmfo_census(W, H, left, prm->census, cl);
    sgmfo_census(W, H, right, prm->census, cr);
    sgmfo_hamming(W, H, D, cl, cr, sgmfo_census_bits(prm->census), hv);
    if (prm->semidense)
        sgmfo_semidense(W, H, D, dbar, hv, prm->ts, prm->rs, dhat);
    else
        memcpy(dhat, dbar, n * sizeof(int16_t));
    sgmfo_ddc(W, H, D, hv, dhat, prm->q1, prm->q2, prm->alpha_num, prm->alpha_den, cv);
    if (dump_cost) memcpy(dump_cost, cv, nv * sizeof(int32_t));
    /* hv is no longer needed: reuse it for S */
    if (sgmfo_aggregate(W, H, D, cv, prm->p1, prm->p2, prm->num_paths, hv) != 0) goto out;
    sgmfo_wta(W, H, D, hv, dstar, dprime);
    sgmfo_consistency(W, H, dstar, dprime, dbar, prm->tc, prm->rc, prm->lr_max_diff,
                      prm->consistency, out);
    if (prm->subpixel) {
        int16_t *dsub = (int16_t *)malloc(n * sizeof(int16_t));
        if (!dsub) goto out;
        sgmfo_subpixel(W, H, D, hv, dstar, dsub);
        for (size_t p = 0; p < n; ++p)
            if (out[p] != SGMFO_INVALID) out[p] = dsub[p];
        free(dsub);
    }
    if (dump_dbar) memcpy(dump_dbar, dbar, n * sizeof(int16_t));
    if (dump_cl) memcpy(dump_cl, cl, n * sizeof(uint64_t));
    if (dump_cr) memcpy(dump_cr, cr, n * sizeof(uint64_t));
    if (dump_dhat) memcpy(dump_dhat, dhat, n * sizeof(int16_t));
    if (dump_sum) memcpy(dump_sum, hv, nv * sizeof(int32_t));
    if (dump_dstar) memcpy(dump_dstar, dstar, n * sizeof(int16_t));
    if (dump_dprime) memcpy(dump_dprime, dprime, n * sizeof(int16_t));
    rc = 0;
out:
    free(dbar); free(dhat); free(dstar); free(dprime);
    free(cl); free(cr); free(hv); free(cv);
    return rc;
}

/* ======================================================================== */
/* Banded SGM.  NOT part of the paper: the method restricted to a disparity
 * band per pixel, the form a learned band proposal drives.  Pixel p keeps the
 * disparities [lo_p, lo_p + B) (clipped to [0, D-1]); every quantity of the
 * method is defined on the band only:
 *   L_r(p, d) = C(p, d) + min{ L_r(p-r, d), L_r(p-r, d-1) + P1,
 *                              L_r(p-r, d+1) + P1, m + P2 } - m,
 *   m = min over the band of p - r of L_r(p - r, k),
 * where a term L_r(p - r, d') is left out when d' is outside the band of
 * p - r (as Eq. 2 leaves out d-1 at d = 0).  This is Eq. 2 read as what it
 * is, the exact dynamic program of the chain energy of Eq. 1: with the
 * labels of every pixel restricted to its band, the best predecessor label
 * of d is any label of the band of p - r, so d-1 and d+1 enter wherever
 * they lie in the band of p - r, whether or not they lie in the band of p.
 * S(p, d) = sum_r L_r(p, d) on the band of
 * p; d*_p = argmin over the band of p; d'(x') = argmin over the d with
 * x' + d < W and d in the band of (x' + d, y) of S(x' + d, y, d), or invalid
 * (-1) when there is none; the stereo term of Eq. 6 needs a valid d'.
 * With lo = 0 and B >= D this is exactly the plain method.  Volumes are full
 * size (H x W x D); cells outside a pixel's band hold SGMFO_ABSENT. */
#define SGMFO_ABSENT (1 << 29)

static int band_hi_(int lo, int B, int D) { return lo + B < D ? lo + B : D; }   /* exclusive */

void sgmfo_path_banded(int W, int H, int D, int B, const int16_t *lo, const int32_t *cv, int p1,
                       int p2, int rx, int ry, int32_t *lv)
{
    for (int iy = 0; iy < H; ++iy) {
        int y = ry >= 0 ? iy : H - 1 - iy;
        for (int ix = 0; ix < W; ++ix) {
            int x = rx >= 0 ? ix : W - 1 - ix;
            size_t pi = (size_t)y * W + x, o = pi * D;
            const int a = lo[pi], ae = band_hi_(a, B, D);
            for (int d = 0; d < D; ++d) lv[o + d] = SGMFO_ABSENT;
            int px = x - rx, py = y - ry;
            if (px < 0 || px >= W || py < 0 || py >= H) {
                for (int d = a; d < ae; ++d) lv[o + d] = cv[o + d];
                continue;
            }
            size_t qi = (size_t)py * W + px, po = qi * D;
            const int b = lo[qi], be = band_hi_(b, B, D);
            int m = 0x7fffffff;
            for (int k = b; k < be; ++k)
                if (lv[po + k] < m) m = lv[po + k];
            for (int d = a; d < ae; ++d) {
                int best = m + p2;
                if (d >= b && d < be && lv[po + d] < best) best = lv[po + d];
                if (d - 1 >= b && d - 1 < be && lv[po + d - 1] + p1 < best) best = lv[po + d - 1] + p1;
                if (d + 1 >= b && d + 1 < be && lv[po + d + 1] + p1 < best) best = lv[po + d + 1] + p1;
                lv[o + d] = cv[o + d] + best - m;
            }
        }
    }
}

int sgmfo_aggregate_banded(int W, int H, int D, int B, const int16_t *lo, const int32_t *cv, int p1,
                           int p2, int num_paths, int32_t *sv)
{
    size_t n = (size_t)W * H * D;
    int32_t *lv = (int32_t *)malloc(n * sizeof(int32_t));
    if (lv == NULL) return -1;
    for (size_t j = 0; j < n; ++j) sv[j] = SGMFO_ABSENT;
    for (size_t pi = 0; pi < (size_t)W * H; ++pi)
        for (int d = lo[pi]; d < band_hi_(lo[pi], B, D); ++d) sv[pi * D + d] = 0;
    for (int i = 0; i < num_paths; ++i) {
        sgmfo_path_banded(W, H, D, B, lo, cv, p1, p2, kDirs[i][0], kDirs[i][1], lv);
        for (size_t pi = 0; pi < (size_t)W * H; ++pi)
            for (int d = lo[pi]; d < band_hi_(lo[pi], B, D); ++d) sv[pi * D + d] += lv[pi * D + d];
    }
    free(lv);
    return 0;
}

void sgmfo_wta_banded(int W, int H, int D, int B, const int16_t *lo, const int32_t *sv,
                      int16_t *dstar, int16_t *dprime)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t pi = (size_t)y * W + x;
            const int32_t *s = sv + pi * D;
            int bd = lo[pi];
            for (int d = lo[pi] + 1; d < band_hi_(lo[pi], B, D); ++d)
                if (s[d] < s[bd]) bd = d;
            dstar[pi] = (int16_t)bd;
        }
    for (int y = 0; y < H; ++y)
        for (int xr = 0; xr < W; ++xr) {
            int bd = SGMFO_INVALID, bs = 0x7fffffff;
            for (int d = 0; d < D && xr + d < W; ++d) {
                size_t pi = (size_t)y * W + xr + d;
                if (d < lo[pi] || d >= band_hi_(lo[pi], B, D)) continue;
                if (sv[pi * D + d] < bs) {
                    bs = sv[pi * D + d];
                    bd = d;
                }
            }
            dprime[(size_t)y * W + xr] = (int16_t)bd;
        }
}

/* The pipeline of sgmfo_compute with the aggregation, WTA and check on the
 * bands (lo: H x W band starts).  dump_sum receives the banded S. */
int sgmfo_compute_banded(const sgmfo_params *prm, int W, int H, int D, int B, const int16_t *lo,
                         const uint8_t *left, const uint8_t *right, const float *lidar,
                         int16_t *out, int32_t *dump_sum, int16_t *dump_dstar, int16_t *dump_dprime)
{
    size_t n = (size_t)W * H, nv = n * (size_t)D;
    int16_t *dbar = (int16_t *)malloc(n * sizeof(int16_t));
    int16_t *dhat = (int16_t *)malloc(n * sizeof(int16_t));
    int16_t *dstar = (int16_t *)malloc(n * sizeof(int16_t));
    int16_t *dprime = (int16_t *)malloc(n * sizeof(int16_t));
    uint64_t *cl = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *cr = (uint64_t *)malloc(n * sizeof(uint64_t));
    int32_t *hv = (int32_t *)malloc(nv * sizeof(int32_t));
    int32_t *cv = (int32_t *)malloc(nv * sizeof(int32_t));
    int rc = -1;
    if (!dbar || !dhat || !dstar || !dprime || !cl || !cr || !hv || !cv) goto out;
    sgmfo_lidar(W, H, D, lidar, dbar);
    sgmfo_census(W, H, left, prm->census, cl);
    sgmfo_census(W, H, right, prm->census, cr);
    sgmfo_hamming(W, H, D, cl, cr, sgmfo_census_bits(prm->census), hv);
    if (prm->semidense)
        sgmfo_semidense(W, H, D, dbar, hv, prm->ts, prm->rs, dhat);
    else
        memcpy(dhat, dbar, n * sizeof(int16_t));
    sgmfo_ddc(W, H, D, hv, dhat, prm->q1, prm->q2, prm->alpha_num, prm->alpha_den, cv);
    if (sgmfo_aggregate_banded(W, H, D, B, lo, cv, prm->p1, prm->p2, prm->num_paths, hv) != 0) goto out;
    sgmfo_wta_banded(W, H, D, B, lo, hv, dstar, dprime);
    consistency_(W, H, dstar, dprime, dbar, prm->tc, prm->rc, prm->lr_max_diff, prm->consistency, 1, out);
    if (dump_sum) memcpy(dump_sum, hv, nv * sizeof(int32_t));
    if (dump_dstar) memcpy(dump_dstar, dstar, n * sizeof(int16_t));
    if (dump_dprime) memcpy(dump_dprime, dprime, n * sizeof(int16_t));
    rc = 0;
out:
    free(dbar); free(dhat); free(dstar); free(dprime);
    free(cl); free(cr); free(hv); free(cv);
    return rc;
}
