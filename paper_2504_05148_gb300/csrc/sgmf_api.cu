// sgmf_api.cu -- the C ABI (include/sgmf.h): contexts, parameter validation,
// scratch ownership, stream handling and the launch sequence of Fig. 1.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sgmf.h"
#include "sgmf_internal.cuh"

using namespace sgmf;

struct sgmf_ctx {
  int device = 0;
  int nb = 1;                  // frames the buffers hold (batch capacity)
  int front_n = 0;             // frames whose front half (sgmf_compute_front) awaits the back half
  KParams k{};
  sgmf_params prm{};
  cudaStream_t stream = nullptr;
  Buffers b{};
  CUtensorMap mapL;   // 64-byte aligned by its declaration
  CUtensorMap mapR;
  bool spill8 = true;
  bool sweep_ok = false;       // the row-synchronous sweep can run this shape on this device (8 paths)
  int sweep_slots = 0;         // sweep clusters the device holds at once
  size_t spill_bytes = 0;
  // with the sweep, a batch goes through in parts: part i's row kernel and
  // check run on this second stream while part i + 1 is in the sweep
  static constexpr int kMaxParts = 8;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_part[kMaxParts] = {};
  cudaEvent_t ev_rows = nullptr, ev_in = nullptr;
  size_t bytes = 0;
  std::string err;
  // device staging for sgmf_compute_host
  uint8_t *st_left = nullptr, *st_right = nullptr;
  float *st_lidar = nullptr;
  int16_t *st_out = nullptr;
  // profiling: an event pair around every launch, on the launching stream
  struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
  };
  bool profiling = false;
  std::vector<cudaEvent_t> ev;     // pool, reused by every compute
  int evused = 0;
  std::vector<ProfRec> recs;
  bool computed = false;
  int last_n = 0;
  bool debug = false;
};

static thread_local std::string g_create_err;

std::mutex &sgmf::setup_mutex() {
  static std::mutex mu;
  return mu;
}

cudaError_t sgmf::sm_count(int *out) {
  static bool done[64] = {};
  static int sms[64] = {};
  int dev = 0;
  cudaError_t e = once_per_device(done, [](int d) { return cudaDeviceGetAttribute(&sms[d], cudaDevAttrMultiProcessorCount, d); });
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) *out = sms[dev];
  return e;
}

static sgmf_status fail(sgmf_ctx *c, sgmf_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_create_err = buf;
  return s;
}

#define CUDA_TRY(c, call)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail((c), e_ == cudaErrorMemoryAllocation ? SGMF_ERR_OOM : SGMF_ERR_CUDA, "%s: %s", \
                  #call, cudaGetErrorString(e_));                                               \
  } while (0)

extern "C" void sgmf_default_params(sgmf_params *p) {
  if (!p) return;
  p->p1 = 10;
  p->p2 = 120;
  p->q1 = 5;
  p->q2 = 160;
  p->alpha_num = 7;
  p->alpha_den = 10;
  p->ts = 2;
  p->rs = 6;
  p->tc = 2;
  p->rc = 20;
  p->lr_max_diff = 1;
  p->census = SGMF_CENSUS_CS9X7;
  p->semidense = 1;
  p->consistency = SGMF_CHECK_STEREO_LIDAR;
  p->num_paths = 8;
  p->subpixel = 0;
}

extern "C" const char *sgmf_status_string(sgmf_status s) {
  switch (s) {
    case SGMF_OK: return "SGMF_OK";
    case SGMF_ERR_ARG: return "SGMF_ERR_ARG";
    case SGMF_ERR_PARAM: return "SGMF_ERR_PARAM";
    case SGMF_ERR_SHAPE: return "SGMF_ERR_SHAPE";
    case SGMF_ERR_OOM: return "SGMF_ERR_OOM";
    case SGMF_ERR_CUDA: return "SGMF_ERR_CUDA";
    case SGMF_ERR_TIMEOUT: return "SGMF_ERR_TIMEOUT";
  }
  return "SGMF_UNKNOWN";
}

static int census_bits(int kind) { return kind == SGMF_CENSUS_9X7 ? 62 : 31; }

// largest joint cost of Eq. 4 under the integer reading
static long max_cost(const sgmf_params &p) {
  const int nb = census_bits(p.census);
  long mx = nb;   // no prior: C-bar = H
  const long qs[3] = {0, p.q1, p.q2};
  for (int h = 0; h <= nb; ++h)
    for (long q : qs) {
      const long v = ((long)(p.alpha_den - p.alpha_num) * h + (long)p.alpha_num * q + p.alpha_den / 2) /
                     p.alpha_den;
      if (v > mx) mx = v;
    }
  return mx;
}

sgmf_status sgmf::validate_params(const sgmf_params &p, std::string &why) {
  char buf[256];
  auto bad = [&](const char *m) {
    why = m;
    return SGMF_ERR_PARAM;
  };
  if (p.p1 < 0 || p.p2 < p.p1 || p.p2 > 2048) return bad("need 0 <= p1 <= p2 <= 2048");
  if (p.q1 < 0 || p.q2 < p.q1 || p.q2 > 1000000) return bad("need 0 <= q1 <= q2 (Sec. IV-A)");
  if (p.alpha_den < 1 || p.alpha_den > 65536 || p.alpha_num < 0 || p.alpha_num > p.alpha_den)
    return bad("need 0 <= alpha_num <= alpha_den, 1 <= alpha_den <= 65536");
  if (p.ts < 0 || p.ts > 65535 || p.rs < 0 || p.rs > 255) return bad("need 0 <= ts <= 65535 and 0 <= rs <= 255");
  if (p.tc < 0 || p.tc > 65535 || p.rc < 0 || p.rc > 255) return bad("need 0 <= tc <= 65535 and 0 <= rc <= 255");
  if (p.lr_max_diff < 0 || p.lr_max_diff > 65535) return bad("need 0 <= lr_max_diff <= 65535");
  if (p.census != SGMF_CENSUS_CS9X7 && p.census != SGMF_CENSUS_9X7) return bad("unknown census kind");
  if (p.semidense != 0 && p.semidense != 1) return bad("semidense must be 0 or 1");
  if (p.consistency < 0 || p.consistency > 3) return bad("unknown consistency mode");
  if (p.num_paths != 4 && p.num_paths != 8) return bad("num_paths must be 4 or 8");
  if (p.subpixel != 0 && p.subpixel != 1) return bad("subpixel must be 0 or 1");
  const long mc = max_cost(p);
  if (mc > 255) {
    snprintf(buf, sizeof buf, "largest joint cost %ld exceeds 255 (uint8 cost volume)", mc);
    why = buf;
    return SGMF_ERR_PARAM;
  }
  return SGMF_OK;
}

static void apply_params(sgmf_ctx *c, const sgmf_params &p) {
  c->prm = p;
  KParams &k = c->k;
  k.p1 = p.p1;
  k.p2 = p.p2;
  k.q1 = p.q1;
  k.q2 = p.q2;
  k.a = p.alpha_num;
  k.b = p.alpha_den;
  k.ts = p.ts;
  k.rs = p.rs;
  k.tc = p.tc;
  k.rc = p.rc;
  k.lr = p.lr_max_diff;
  k.census = p.census;
  k.semidense = p.semidense;
  k.consistency = p.consistency;
  k.num_paths = p.num_paths;
  k.subpixel = p.subpixel;
  k.nbits = census_bits(p.census);
  c->spill8 = max_cost(p) + p.p2 <= 255;
}

static void free_all(sgmf_ctx *c) {
  void *ptrs[] = {c->b.imgL, c->b.imgR, c->b.dbar, c->b.dhat, c->b.dstar, c->b.dprime, c->b.dsub, c->b.censL,
                  c->b.censR, c->b.boxS, c->b.boxC, c->b.boxTmp, c->b.cost, c->b.part[0],
                  c->b.part[1], c->b.part[2], c->b.spill, c->b.dbg_sum, c->b.band_lo, c->b.err, c->st_left,
                  c->st_right, c->st_lidar, c->st_out};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  c->ev.clear();
  for (int i = 0; i < sgmf_ctx::kMaxParts; ++i) {
    if (c->ev_part[i]) cudaEventDestroy(c->ev_part[i]);
    c->ev_part[i] = nullptr;
  }
  for (cudaEvent_t *e : {&c->ev_rows, &c->ev_in}) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  if (c->side) cudaStreamDestroy(c->side);
  c->side = nullptr;
}

// test hook (sgmf_debug_fail_alloc): allocations until the injected failure
static thread_local int g_fail_alloc = 0;

extern "C" void sgmf_debug_fail_alloc(int n) { g_fail_alloc = n > 0 ? n : 0; }

template <typename T>
static cudaError_t dalloc(sgmf_ctx *c, T **p, size_t bytes) {
  if (g_fail_alloc > 0 && --g_fail_alloc == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;     // injected: cudaMalloc is not called
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
  if (e == cudaSuccess) c->bytes += bytes;
  return e;
}

extern "C" sgmf_status sgmf_create(int width, int height, int max_disp, sgmf_ctx **out) {
  return sgmf_create_batched(width, height, max_disp, 1, out);
}

// the side stream of the row kernels and checks of a batch in parts, at the
// priority of a default stream (kSidePriority = 1, above it, was measured:
// 8.14-8.21 against 8.12 ms for 32 KITTI frames -- the row kernels got ahead,
// the sweep fell behind by as much)
static cudaError_t side_stream(cudaStream_t *s) {
  constexpr int kSidePriority = 0;
  int least = 0, greatest = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e != cudaSuccess) return e;
  return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, kSidePriority ? greatest : least);
}

static sgmf_status create_ctx(int width, int height, int max_disp, int max_batch, int band, sgmf_ctx **out) {
  if (!out) return fail(nullptr, SGMF_ERR_ARG, "sgmf_create: out is NULL");
  *out = nullptr;
  if (width < 1 || height < 1 || width > kMaxDim || height > kMaxDim || max_disp < 1 || max_disp > kMaxDisp)
    return fail(nullptr, SGMF_ERR_SHAPE,
                "sgmf_create: need 1 <= width, height <= %d and 1 <= max_disp <= %d (got %d x %d, D=%d)",
                kMaxDim, kMaxDisp, width, height, max_disp);
  if (max_batch < 1 || max_batch > 4096)
    return fail(nullptr, SGMF_ERR_SHAPE, "sgmf_create_batched: need 1 <= max_batch <= 4096 (got %d)", max_batch);
  sgmf_ctx *c = new (std::nothrow) sgmf_ctx();
  if (!c) return fail(nullptr, SGMF_ERR_OOM, "sgmf_create: host allocation failed");
  cudaGetDevice(&c->device);
  c->nb = max_batch;
  KParams &k = c->k;
  k.W = width;
  k.H = height;
  k.D = max_disp;
  k.DPL = max_disp <= 64 ? 2 : max_disp <= 128 ? 4 : max_disp <= 192 ? 6 : 8;
  k.Dp = 32 * k.DPL;
  k.MW = k.Dp / 32;          // presence-mask words cover [0, D)
  k.band = band;
  if (band) {                // lanes and volumes hold the band only
    k.Dp = band;
    k.DPL = band / 32;
    k.tw = (width + kBandTile - 1) / kBandTile;
    k.th = (height + kBandTile - 1) / kBandTile;
  }
  k.pitch = (width + 15) / 16 * 16;
  k.line_warps = 4;
  k.cost_px = 128;
  k.wait_census = kWaitLimit;
  k.sweep = 0;
  k.parts = 1;
  sgmf_params def;
  sgmf_default_params(&def);
  apply_params(c, def);

  const size_t n = (size_t)width * height * max_batch, nv = n * k.Dp;   // all frames
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  A(dalloc(c, &c->b.imgL, (size_t)k.pitch * height * max_batch));
  A(dalloc(c, &c->b.imgR, (size_t)k.pitch * height * max_batch));
  A(dalloc(c, &c->b.dbar, n * 2));
  A(dalloc(c, &c->b.dhat, n * 2));
  A(dalloc(c, &c->b.dstar, n * 2));
  A(dalloc(c, &c->b.dprime, n * 2));
  A(dalloc(c, &c->b.dsub, n * 2));
  A(dalloc(c, reinterpret_cast<uint64_t **>(&c->b.censL), n * 8));
  A(dalloc(c, reinterpret_cast<uint64_t **>(&c->b.censR), n * 8));
  A(dalloc(c, &c->b.boxS, n * 4 * k.MW));
  A(dalloc(c, &c->b.boxC, n * 4 * k.MW));
  A(dalloc(c, &c->b.boxTmp, n * 4 * k.MW));
  A(dalloc(c, &c->b.cost, nv));
  for (int i = 0; i < 3; ++i) A(dalloc(c, &c->b.part[i], nv * 2));
  c->spill_bytes = 4 * nv * 2;
  A(dalloc(c, reinterpret_cast<uint16_t **>(&c->b.spill), c->spill_bytes));
  if (band) {
    A(dalloc(c, &c->b.band_lo, (size_t)k.tw * k.th * max_batch * 2));
  }
  A(dalloc(c, &c->b.err, sizeof(int)));
  if (e == cudaSuccess) e = cudaMemset(c->b.err, 0, sizeof(int));
  if (e != cudaSuccess) {
    sgmf_status s = fail(nullptr, e == cudaErrorMemoryAllocation ? SGMF_ERR_OOM : SGMF_ERR_CUDA,
                         "sgmf_create: device allocation of %zu bytes failed: %s", c->bytes,
                         cudaGetErrorString(e));
    free_all(c);
    delete c;
    cudaGetLastError();
    return s;
  }
  if (make_image_tmap(&c->mapL, c->b.imgL, width, height, k.pitch, max_batch, kCenBoxW, kCenBoxH) != 0 ||
      make_image_tmap(&c->mapR, c->b.imgR, width, height, k.pitch, max_batch, kCenBoxW, kCenBoxH) != 0) {
    free_all(c);
    delete c;
    return fail(nullptr, SGMF_ERR_CUDA, "sgmf_create: cuTensorMapEncodeTiled failed");
  }
  {
    // whether the row-synchronous sweep can run this shape (8 paths); the
    // line kernels stay the default, the sweep is a tuning choice
    KParams kk = k;
    kk.num_paths = 8;
    c->k.sweep_cs = agg_sweep_plan(kk, c->nb, &c->sweep_slots);
    c->sweep_ok = c->k.sweep_cs > 0;
    bool ok = !(c->sweep_ok && c->nb >= 2) ||
              (side_stream(&c->side) == cudaSuccess &&
               cudaEventCreateWithFlags(&c->ev_rows, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) == cudaSuccess);
    for (int i = 0; ok && c->side && i < sgmf_ctx::kMaxParts; ++i)
      ok = cudaEventCreateWithFlags(&c->ev_part[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      c->sweep_slots = 0;        // no parts: everything on the context's stream
    }
  }
  *out = c;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_create_batched(int width, int height, int max_disp, int max_batch, sgmf_ctx **out) {
  return create_ctx(width, height, max_disp, max_batch, 0, out);
}

extern "C" sgmf_status sgmf_create_banded(int width, int height, int max_disp, int band, int max_batch,
                                          sgmf_ctx **out) {
  if (out) *out = nullptr;
  if (band != 64 && band != 128)
    return fail(nullptr, SGMF_ERR_SHAPE, "sgmf_create_banded: band must be 64 or 128 (got %d)", band);
  if (max_disp < band)
    return fail(nullptr, SGMF_ERR_SHAPE, "sgmf_create_banded: need band <= max_disp (got %d > %d)", band, max_disp);
  return create_ctx(width, height, max_disp, max_batch, band, out);
}

extern "C" void sgmf_destroy(sgmf_ctx *c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_all(c);
  cudaSetDevice(prev);
  delete c;
}

void sgmf::set_noctx_error(const std::string &msg) { g_create_err = msg; }

extern "C" const char *sgmf_last_error(const sgmf_ctx *c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

extern "C" sgmf_status sgmf_set_params(sgmf_ctx *c, const sgmf_params *p) {
  if (!c || !p) return fail(c, SGMF_ERR_ARG, "sgmf_set_params: NULL argument");
  std::string why;
  if (validate_params(*p, why) != SGMF_OK) return fail(c, SGMF_ERR_PARAM, "sgmf_set_params: %s", why.c_str());
  apply_params(c, *p);
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_get_params(const sgmf_ctx *c, sgmf_params *p) {
  if (!c || !p) return SGMF_ERR_ARG;
  *p = c->prm;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_set_gate(sgmf_ctx *c, const int *gate, int run) {
  if (!c) return SGMF_ERR_ARG;
  c->b.gate = gate;
  c->k.gate_run = run;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_set_wait_limit(sgmf_ctx *c, int which, long long polls) {
  if (!c) return SGMF_ERR_ARG;
  if (which != SGMF_WAIT_CENSUS) return fail(c, SGMF_ERR_ARG, "sgmf_set_wait_limit: unknown wait %d", which);
  c->k.wait_census = polls < 0 ? kWaitLimit : (uint32_t)std::min<long long>(polls, 0xffffffffLL);
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_set_stream(sgmf_ctx *c, void *stream) {
  if (!c) return SGMF_ERR_ARG;
  c->stream = static_cast<cudaStream_t>(stream);
  return SGMF_OK;
}

static bool need_boxc(const KParams &k) { return k.consistency == SGMF_CHECK_STEREO_LIDAR || k.consistency == SGMF_CHECK_LIDAR; }

// the sweep runs when the tuning asks for it and the context allows it
static bool use_sweep(const sgmf_ctx *c) { return c->k.sweep && c->k.num_paths == 8 && c->sweep_ok; }

// Frames per part when a sweep batch of n frames goes through in parts (0:
// one part).  A part's row kernel and check run on the side stream beside
// the next part's sweep, filling the SMs (and the register room) the sweep
// clusters leave.  Every part but the last is one wave of sweep clusters
// (2 m cluster jobs, the resident count or its smallest even multiple), so
// the parts add no wave; at most kMaxParts parts.
static int sweep_part(const sgmf_ctx *c, int n) {
  if (!c->k.parts || !c->side || c->sweep_slots < 1 || n < 2) return 0;
  int m = c->sweep_slots % 2 == 0 ? c->sweep_slots / 2 : c->sweep_slots;   // 2 m % slots == 0
  if (m >= n) return 0;
  while ((n + m - 1) / m > sgmf_ctx::kMaxParts) m *= 2;
  return m;
}

// parameters of the aggregation launches: the sweep flag as it will run
static KParams agg_params(const sgmf_ctx *c) {
  KParams k = c->k;
  k.sweep = use_sweep(c) ? 1 : 0;
  return k;
}

// launches of the front stages (ingest, census, box-OR row pass and, for
// Eq. 5, its column pass, cost with Eq. 5 inside)
static int front_launches(const KParams &k) {
  return 3 + ((k.semidense || need_boxc(k)) ? 1 : 0) + (k.semidense ? 1 : 0);
}

extern "C" int sgmf_launches_per_compute(const sgmf_ctx *c) {
  if (!c) return 0;
  // front stages, one line launch per family (one sweep launch for all six directions), rows, consistency
  // (a sweep batch in parts launches the sweep, rows and check once per part; counted for a full batch)
  const int agg = (c->k.num_paths == 8 ? (use_sweep(c) ? 1 : 3) : 1) + 2;
  int parts = 1;
  if (use_sweep(c) && sweep_part(c, c->nb) > 0) {
    const int m = sweep_part(c, c->nb);
    parts = (c->nb + m - 1) / m;
  }
  // banded: the front half runs Eq. 5 on its own (+1) and the back half clamps the bands (+1)
  return front_launches(c->k) + agg * parts + (c->k.band ? 1 + (c->k.semidense ? 1 : 0) : 0);
}

// an event of the pool (null when none can be created: that launch goes untimed)
static cudaEvent_t prof_event(sgmf_ctx *c) {
  if (c->evused >= (int)c->ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    c->ev.push_back(e);
  }
  return c->ev[c->evused++];
}

// start / end of a timed launch on stream s (profiling on)
static int prof_begin(sgmf_ctx *c, const char *name, cudaStream_t s) {
  if (!c->profiling) return -1;
  cudaEvent_t a = prof_event(c), b = prof_event(c);
  if (!a || !b) return -1;
  cudaEventRecord(a, s);
  c->recs.push_back({name, a, b});
  return (int)c->recs.size() - 1;
}

static void prof_end(sgmf_ctx *c, int r, cudaStream_t s) {
  if (r >= 0) cudaEventRecord(c->recs[r].b, s);
}

static void prof_reset(sgmf_ctx *c) {
  c->recs.clear();
  c->evused = 0;
}

#define LAUNCH_TRY(c, call)                                                          \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail((c), SGMF_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

// a launch between the events of one profiling record
#define TIMED(c, name, s, call)                     \
  do {                                              \
    const int r_ = prof_begin((c), (name), (s));    \
    LAUNCH_TRY((c), (call));                        \
    prof_end((c), r_, (s));                         \
  } while (0)

// The stages before aggregation (ingest, census, box-OR, semidense and,
// with `cost`, the cost volume) for frames [f0, f0 + nf) on stream s; the
// inputs are the call's frame-0 pointers.
static sgmf_status front_stages(sgmf_ctx *c, int f0, int nf, const uint8_t *left, const uint8_t *right,
                                const float *lidar, bool cost, cudaStream_t s) {
  const KParams &k = c->k;
  const size_t px = (size_t)k.W * k.H;
  const Buffers bp = frame_view(k, c->b, f0);
  TIMED(c, "ingest", s, launch_ingest(k, bp, nf, left + f0 * px, right + f0 * px, lidar ? lidar + f0 * px : nullptr, s));
  TIMED(c, "census", s, launch_census(k, bp, nf, f0, &c->mapL, &c->mapR, s));
  if (k.semidense || need_boxc(k)) {
    // both windows' row pass at once; the column pass for r_s (Eq. 5) into
    // boxS, from the row results of frames [f0, f0 + nf) in their own part
    // of boxTmp; the r_c row ORs (Eq. 6) stay in boxC for the check.  (On
    // the side stream beside the census it saved 0.01 ms of 8.18 for 32
    // KITTI frames: the two run one after the other all the same.)
    TIMED(c, "boxor", s, launch_boxor(k, nf, bp.dbar, c->b.boxTmp + (size_t)f0 * k.MW * px,
                                      k.semidense ? bp.boxS : nullptr, need_boxc(k) ? bp.boxC : nullptr, s,
                                      bp.gate));
  }
  // with the cost volume, Eq. 5 runs inside the cost kernel (its candidates'
  // right-census words are staged there anyway); alone for the banded front half
  if (k.semidense && !cost) TIMED(c, "semidense", s, launch_semidense(k, bp, nf, s));
  if (cost) TIMED(c, "cost", s, launch_cost(k, bp, nf, s));
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_compute_batch(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                                          const float *lidar, int16_t *out) {
  if (!c) return SGMF_ERR_ARG;
  if (!left || !right || !out) return fail(c, SGMF_ERR_ARG, "sgmf_compute: NULL image or output pointer");
  if (n < 1 || n > c->nb)
    return fail(c, SGMF_ERR_ARG, "sgmf_compute_batch: need 1 <= n <= %d frames (got %d)", c->nb, n);
  if (c->k.band) return fail(c, SGMF_ERR_ARG, "sgmf_compute: a banded context needs sgmf_compute_banded");
  const KParams &k = c->k;
  const size_t px = (size_t)k.W * k.H;
  cudaStream_t s = c->stream;
  prof_reset(c);
  const KParams ka = agg_params(c);
  const int m = ka.sweep ? sweep_part(c, n) : 0;
  if (m > 0) {
    // Parts of m frames after the front stages of all n: part i's sweep on
    // the context's stream, then its row kernel and check on the side
    // stream while part i + 1 is in the sweep; the context's stream goes on
    // after the last part's check.  (Running the later parts' front stages
    // on the side stream beside the first part's sweep was measured twice
    // and gave nothing: 8.17-8.24 against 8.20 ms for 32 KITTI frames, and
    // 3 % slower at 64; the sweep slows by what the front stages save.)
    sgmf_status st = front_stages(c, 0, n, left, right, lidar, true, s);
    if (st != SGMF_OK) return st;
    for (int i = 0, f0 = 0; f0 < n; ++i, f0 += m) {
      const int nf = std::min(m, n - f0);
      const Buffers bp = frame_view(k, c->b, f0);
      TIMED(c, "agg_sweep", s, launch_agg_sweep(ka, bp, nf, s));
      CUDA_TRY(c, cudaEventRecord(c->ev_part[i], s));
      CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_part[i], 0));
      TIMED(c, "agg_rows_wta", c->side, launch_agg_rows(ka, bp, nf, c->spill8, c->side));
      TIMED(c, "consistency", c->side, launch_consistency(k, bp, nf, out + f0 * px, c->side));
    }
    CUDA_TRY(c, cudaEventRecord(c->ev_rows, c->side));
    CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_rows, 0));
  } else {
    sgmf_status st = front_stages(c, 0, n, left, right, lidar, true, s);
    if (st != SGMF_OK) return st;
    if (ka.sweep)
      TIMED(c, "agg_sweep", s, launch_agg_sweep(ka, c->b, n, s));
    else
      TIMED(c, "agg_lines", s, launch_agg_lines(ka, c->b, n, c->spill8, s));
    TIMED(c, "agg_rows_wta", s, launch_agg_rows(ka, c->b, n, c->spill8, s));
    TIMED(c, "consistency", s, launch_consistency(k, c->b, n, out, s));
  }
  c->computed = true;
  c->last_n = n;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_compute(sgmf_ctx *c, const uint8_t *left, const uint8_t *right, const float *lidar,
                                    int16_t *out) {
  return sgmf_compute_batch(c, 1, left, right, lidar, out);
}

extern "C" sgmf_status sgmf_sync(sgmf_ctx *c) {
  if (!c) return SGMF_ERR_ARG;
  cudaError_t e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(c, SGMF_ERR_CUDA, "sgmf_sync: %s", cudaGetErrorString(e));
  int flag = 0;
  CUDA_TRY(c, cudaMemcpy(&flag, c->b.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag != 0) {
    CUDA_TRY(c, cudaMemset(c->b.err, 0, sizeof(int)));
    if (flag == kErrTimeout)
      return fail(c, SGMF_ERR_TIMEOUT, "sgmf_sync: a bounded device wait gave up (TMA copy did not land)");
    return fail(c, SGMF_ERR_CUDA, "sgmf_sync: device error word %d", flag);
  }
  return SGMF_OK;
}

// the host entry point's work, enqueued on the context's stream (no wait)
static sgmf_status enqueue_host_batch(sgmf_ctx *c, int nf, const uint8_t *left, const uint8_t *right,
                                      const float *lidar, int16_t *out) {
  if (!c) return SGMF_ERR_ARG;
  if (!left || !right || !out) return fail(c, SGMF_ERR_ARG, "sgmf_compute_host: NULL image or output pointer");
  if (nf < 1 || nf > c->nb)
    return fail(c, SGMF_ERR_ARG, "sgmf_compute_host_batch: need 1 <= n <= %d frames (got %d)", c->nb, nf);
  const size_t cap = (size_t)c->k.W * c->k.H * c->nb;
  const size_t n = (size_t)c->k.W * c->k.H * nf;
  if (!c->st_left) {
    // the four staging buffers, all or none
    uint8_t *l = nullptr, *r = nullptr;
    float *li = nullptr;
    int16_t *o = nullptr;
    const size_t held = c->bytes;
    cudaError_t e = dalloc(c, &l, cap);
    if (e == cudaSuccess) e = dalloc(c, &r, cap);
    if (e == cudaSuccess) e = dalloc(c, &li, cap * 4);
    if (e == cudaSuccess) e = dalloc(c, &o, cap * 2);
    if (e != cudaSuccess) {
      for (void *p : {(void *)l, (void *)r, (void *)li, (void *)o})
        if (p) cudaFree(p);
      c->bytes = held;
      cudaGetLastError();
      return fail(c, e == cudaErrorMemoryAllocation ? SGMF_ERR_OOM : SGMF_ERR_CUDA,
                  "sgmf_compute_host: staging allocation failed: %s", cudaGetErrorString(e));
    }
    c->st_left = l;
    c->st_right = r;
    c->st_lidar = li;
    c->st_out = o;
  }
  cudaStream_t s = c->stream;
  CUDA_TRY(c, cudaMemcpyAsync(c->st_left, left, n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(c, cudaMemcpyAsync(c->st_right, right, n, cudaMemcpyHostToDevice, s));
  if (lidar) CUDA_TRY(c, cudaMemcpyAsync(c->st_lidar, lidar, n * 4, cudaMemcpyHostToDevice, s));
  sgmf_status st = sgmf_compute_batch(c, nf, c->st_left, c->st_right, lidar ? c->st_lidar : nullptr, c->st_out);
  if (st != SGMF_OK) return st;
  CUDA_TRY(c, cudaMemcpyAsync(out, c->st_out, n * 2, cudaMemcpyDeviceToHost, s));
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_compute_host_batch(sgmf_ctx *c, int nf, const uint8_t *left, const uint8_t *right,
                                               const float *lidar, int16_t *out) {
  const sgmf_status st = enqueue_host_batch(c, nf, left, right, lidar, out);
  return st != SGMF_OK ? st : sgmf_sync(c);
}

extern "C" sgmf_status sgmf_compute_host_batch_async(sgmf_ctx *c, int nf, const uint8_t *left, const uint8_t *right,
                                                     const float *lidar, int16_t *out) {
  return enqueue_host_batch(c, nf, left, right, lidar, out);
}

extern "C" sgmf_status sgmf_compute_host(sgmf_ctx *c, const uint8_t *left, const uint8_t *right,
                                         const float *lidar, int16_t *out) {
  return sgmf_compute_host_batch(c, 1, left, right, lidar, out);
}

extern "C" int sgmf_batch_capacity(const sgmf_ctx *c) { return c ? c->nb : 0; }

extern "C" sgmf_status sgmf_set_debug(sgmf_ctx *c, int enable) {
  if (!c) return SGMF_ERR_ARG;
  if (enable && !c->b.dbg_sum) {
    CUDA_TRY(c, dalloc(c, &c->b.dbg_sum, (size_t)c->k.W * c->k.H * c->k.Dp * 2));
  } else if (!enable && c->b.dbg_sum) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->b.dbg_sum);
    c->bytes -= (size_t)c->k.W * c->k.H * c->k.Dp * 2;
    c->b.dbg_sum = nullptr;
  }
  c->debug = enable != 0;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_debug_stage(sgmf_ctx *c, int stage, void *dst, size_t bytes) {
  if (!c) return SGMF_ERR_ARG;
  if (!dst) return fail(c, SGMF_ERR_ARG, "sgmf_debug_stage: NULL destination");
  const KParams &k = c->k;
  const size_t n = (size_t)k.W * k.H;
  size_t need = 0;
  switch (stage) {
    case SGMF_STAGE_DBAR: case SGMF_STAGE_DHAT: case SGMF_STAGE_DSTAR: case SGMF_STAGE_DPRIME:
    case SGMF_STAGE_DSUB: need = n * 2; break;
    case SGMF_STAGE_CENSUS_L: case SGMF_STAGE_CENSUS_R: need = n * 8; break;
    case SGMF_STAGE_COST: need = n * (k.band ? k.band : k.D); break;
    case SGMF_STAGE_SUM: need = n * (k.band ? k.band : k.D) * 2; break;
    case SGMF_STAGE_BOX_S: case SGMF_STAGE_BOX_C: need = n * 4 * k.MW; break;
    default: return fail(c, SGMF_ERR_ARG, "sgmf_debug_stage: unknown stage %d", stage);
  }
  if (stage == SGMF_STAGE_BOX_S && !k.semidense)
    return fail(c, SGMF_ERR_ARG, "sgmf_debug_stage: BOX_S needs semidense = 1");
  if (stage == SGMF_STAGE_BOX_C && !need_boxc(k))
    return fail(c, SGMF_ERR_ARG, "sgmf_debug_stage: BOX_C needs a consistency mode with the LiDAR check");
  if (bytes < need) return fail(c, SGMF_ERR_ARG, "sgmf_debug_stage: need %zu bytes, got %zu", need, bytes);
  if (stage == SGMF_STAGE_DSUB && !k.subpixel)
    return fail(c, SGMF_ERR_ARG, "sgmf_debug_stage: DSUB needs subpixel = 1");
  if (stage == SGMF_STAGE_SUM && !c->b.dbg_sum)
    return fail(c, SGMF_ERR_ARG, "sgmf_debug_stage: SUM needs sgmf_set_debug(c, 1) before sgmf_compute");
  sgmf_status st = sgmf_sync(c);
  if (st != SGMF_OK) return st;
  switch (stage) {
    case SGMF_STAGE_DBAR: CUDA_TRY(c, cudaMemcpy(dst, c->b.dbar, need, cudaMemcpyDeviceToHost)); break;
    case SGMF_STAGE_DHAT:
      CUDA_TRY(c, cudaMemcpy(dst, k.semidense ? c->b.dhat : c->b.dbar, need, cudaMemcpyDeviceToHost));
      break;
    case SGMF_STAGE_DSTAR: CUDA_TRY(c, cudaMemcpy(dst, c->b.dstar, need, cudaMemcpyDeviceToHost)); break;
    case SGMF_STAGE_DPRIME: CUDA_TRY(c, cudaMemcpy(dst, c->b.dprime, need, cudaMemcpyDeviceToHost)); break;
    case SGMF_STAGE_DSUB: CUDA_TRY(c, cudaMemcpy(dst, c->b.dsub, need, cudaMemcpyDeviceToHost)); break;
    case SGMF_STAGE_BOX_S: CUDA_TRY(c, cudaMemcpy(dst, c->b.boxS, need, cudaMemcpyDeviceToHost)); break;
    case SGMF_STAGE_BOX_C:
      // the pipeline keeps the row ORs only: the column pass of frame 0 into scratch
      LAUNCH_TRY(c, launch_boxor_cols(k, 1, c->b.boxC, c->b.boxTmp, k.rc, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      CUDA_TRY(c, cudaMemcpy(dst, c->b.boxTmp, need, cudaMemcpyDeviceToHost));
      break;
    case SGMF_STAGE_CENSUS_L:
    case SGMF_STAGE_CENSUS_R: {
      const void *src = stage == SGMF_STAGE_CENSUS_L ? c->b.censL : c->b.censR;
      if (k.census == SGMF_CENSUS_9X7) {
        CUDA_TRY(c, cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost));
      } else {
        std::vector<uint32_t> tmp(n);
        CUDA_TRY(c, cudaMemcpy(tmp.data(), src, n * 4, cudaMemcpyDeviceToHost));
        uint64_t *o = static_cast<uint64_t *>(dst);
        for (size_t i = 0; i < n; ++i) o[i] = tmp[i];
      }
      break;
    }
    case SGMF_STAGE_COST:
      CUDA_TRY(c, cudaMemcpy2D(dst, need / n, c->b.cost, k.Dp, need / n, n, cudaMemcpyDeviceToHost));
      break;
    case SGMF_STAGE_SUM:
      if (k.band) {   // banded: [H][W][band], cell j = disparity lo_p + j
        CUDA_TRY(c, cudaMemcpy(dst, c->b.dbg_sum, need, cudaMemcpyDeviceToHost));
        break;
      }
      CUDA_TRY(c, cudaMemcpy2D(dst, (size_t)k.D * 2, c->b.dbg_sum, (size_t)k.Dp * 2, (size_t)k.D * 2, n,
                               cudaMemcpyDeviceToHost));
      break;
  }
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_set_profiling(sgmf_ctx *c, int enable) {
  if (!c) return SGMF_ERR_ARG;
  c->profiling = enable != 0;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_kernel_times(sgmf_ctx *c, const char **names, float *ms, int *n) {
  if (!c || !n) return SGMF_ERR_ARG;
  // the launches of each kernel name summed, names in order of first launch
  std::vector<const char *> nm;
  std::vector<float> tot;
  for (const sgmf_ctx::ProfRec &r : c->recs) {
    float t = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, r.a, r.b));
    size_t j = 0;
    while (j < nm.size() && strcmp(nm[j], r.name) != 0) ++j;
    if (j == nm.size()) {
      nm.push_back(r.name);
      tot.push_back(0.f);
    }
    tot[j] += t;
  }
  const int cap = *n;
  for (int i = 0; i < (int)nm.size() && i < cap; ++i) {
    if (names) names[i] = nm[i];
    if (ms) ms[i] = tot[i];
  }
  *n = (int)nm.size();
  return SGMF_OK;
}

extern "C" size_t sgmf_device_bytes(const sgmf_ctx *c) { return c ? c->bytes : 0; }

// ---- launch tuning -------------------------------------------------------------
static bool valid_tuning(const sgmf_tuning &t) {
  return (t.line_warps == 1 || t.line_warps == 2 || t.line_warps == 4 || t.line_warps == 8) &&
         (t.cost_px == 32 || t.cost_px == 64 || t.cost_px == 128) && (t.sweep == 0 || t.sweep == 1) &&
         (t.parts == 0 || t.parts == 1);
}

extern "C" sgmf_status sgmf_set_tuning(sgmf_ctx *c, const sgmf_tuning *t) {
  if (!c || !t) return fail(c, SGMF_ERR_ARG, "sgmf_set_tuning: NULL argument");
  if (!valid_tuning(*t))
    return fail(c, SGMF_ERR_ARG,
                "sgmf_set_tuning: need line_warps in {1,2,4,8}, cost_px in {32,64,128}, sweep and parts in {0,1}");
  if (t->sweep && !c->sweep_ok)
    return fail(c, SGMF_ERR_ARG, "sgmf_set_tuning: the sweep does not fit this context (a row wider than one "
                                 "cluster holds)");
  c->k.line_warps = t->line_warps;
  c->k.cost_px = t->cost_px;
  c->k.sweep = t->sweep;
  c->k.parts = t->parts;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_get_tuning(const sgmf_ctx *c, sgmf_tuning *t) {
  if (!c || !t) return SGMF_ERR_ARG;
  t->line_warps = c->k.line_warps;
  t->cost_px = c->k.cost_px;
  t->sweep = c->k.sweep;
  t->parts = c->k.parts;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_autotune(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                                     const float *lidar, int16_t *out, int reps, sgmf_tuning *best,
                                     float *best_ms) {
  if (!c) return SGMF_ERR_ARG;
  if (reps < 1 || reps > 100) return fail(c, SGMF_ERR_ARG, "sgmf_autotune: need 1 <= reps <= 100 (got %d)", reps);
  const bool prof = c->profiling;
  c->profiling = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sgmf_status st = SGMF_OK;
  sgmf_tuning keep{c->k.line_warps, c->k.cost_px, c->k.sweep, c->k.parts}, win = keep;
  float win_ms = 0.0f;
  bool have = false;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = fail(c, SGMF_ERR_CUDA, "sgmf_autotune: cudaEventCreate failed");
  }
  // the 4 x 3 line-kernel shapes, then the sweep with each cost shape
  const int warps[4] = {1, 2, 4, 8}, pxs[3] = {32, 64, 128};
  const int ncand = 12 + (c->sweep_ok && c->k.num_paths == 8 ? 3 : 0);
  std::vector<float> t;
  for (int i = 0; i < ncand && st == SGMF_OK; ++i) {
    c->k.sweep = i >= 12;
    c->k.line_warps = i < 12 ? warps[i / 3] : keep.line_warps;
    c->k.cost_px = pxs[i % 3];
    st = sgmf_compute_batch(c, n, left, right, lidar, out);   // warm-up (and first-use attributes)
    t.clear();
    for (int r = 0; r < reps && st == SGMF_OK; ++r) {
      // start each timed run with a cold L2, as a stream of batches finds it:
      // overwrite part of the spill scratch (rewritten by every compute anyway)
      cudaMemsetAsync(c->b.spill, 0, std::min(c->spill_bytes, (size_t)256 << 20), c->stream);
      cudaEventRecord(e0, c->stream);
      st = sgmf_compute_batch(c, n, left, right, lidar, out);
      cudaEventRecord(e1, c->stream);
      if (st != SGMF_OK) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = fail(c, SGMF_ERR_CUDA, "sgmf_autotune: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      t.push_back(ms);
    }
    if (st != SGMF_OK) break;
    st = sgmf_sync(c);
    if (st != SGMF_OK) break;
    std::sort(t.begin(), t.end());
    const float med = t[t.size() / 2];
    if (!have || med < win_ms) {
      have = true;
      win_ms = med;
      win = sgmf_tuning{c->k.line_warps, c->k.cost_px, c->k.sweep, c->k.parts};
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->profiling = prof;
  const sgmf_tuning chosen = st == SGMF_OK ? win : keep;
  c->k.line_warps = chosen.line_warps;
  c->k.cost_px = chosen.cost_px;
  c->k.sweep = chosen.sweep;
  if (st != SGMF_OK) return st;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return SGMF_OK;
}

// ---- banded mode ---------------------------------------------------------------
extern "C" sgmf_status sgmf_compute_front(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                                          const float *lidar) {
  if (!c) return SGMF_ERR_ARG;
  if (!left || !right) return fail(c, SGMF_ERR_ARG, "sgmf_compute_front: NULL image pointer");
  if (!c->k.band) return fail(c, SGMF_ERR_ARG, "sgmf_compute_front: context is not banded (sgmf_create_banded)");
  if (n < 1 || n > c->nb)
    return fail(c, SGMF_ERR_ARG, "sgmf_compute_front: need 1 <= n <= %d frames (got %d)", c->nb, n);
  prof_reset(c);
  const sgmf_status st = front_stages(c, 0, n, left, right, lidar, false, c->stream);
  if (st != SGMF_OK) return st;
  c->front_n = n;   // the caller's band proposal runs before the back half
  return SGMF_OK;
}

extern "C" const int16_t *sgmf_prior_device(const sgmf_ctx *c) {
  if (!c) return nullptr;
  return c->k.semidense ? c->b.dhat : c->b.dbar;
}

extern "C" sgmf_status sgmf_compute_banded_back(sgmf_ctx *c, int n, const int16_t *band_lo, int16_t *out) {
  if (!c) return SGMF_ERR_ARG;
  if (!out || !band_lo) return fail(c, SGMF_ERR_ARG, "sgmf_compute_banded_back: NULL pointer");
  if (!c->k.band) return fail(c, SGMF_ERR_ARG, "sgmf_compute_banded_back: context is not banded");
  if (n < 1 || n != c->front_n)
    return fail(c, SGMF_ERR_ARG, "sgmf_compute_banded_back: needs the %d frames of the last sgmf_compute_front (got %d)",
                c->front_n, n);
  if (c->k.subpixel) return fail(c, SGMF_ERR_PARAM, "sgmf_compute_banded: subpixel must be 0");
  const KParams &k = c->k;
  cudaStream_t s = c->stream;
  TIMED(c, "band_clamp", s, launch_band_clamp(k, c->b, n, band_lo, s));
  TIMED(c, "cost", s, launch_cost_banded(k, c->b, n, s));
  const KParams ka = agg_params(c);
  const int m = ka.sweep ? sweep_part(c, n) : 0;
  if (m > 0) {
    // parts of m frames: part i's row kernel and check on the side stream
    // beside part i + 1's sweep (as in sgmf_compute_batch)
    const size_t px = (size_t)k.W * k.H;
    CUDA_TRY(c, cudaEventRecord(c->ev_in, s));
    CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_in, 0));
    for (int i = 0, f0 = 0; f0 < n; ++i, f0 += m) {
      const int nf = std::min(m, n - f0);
      const Buffers bp = frame_view(k, c->b, f0);
      TIMED(c, "agg_sweep", s, launch_agg_sweep(ka, bp, nf, s));
      CUDA_TRY(c, cudaEventRecord(c->ev_part[i], s));
      CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_part[i], 0));
      TIMED(c, "agg_rows_wta", c->side, launch_agg_rows(ka, bp, nf, c->spill8, c->side));
      TIMED(c, "consistency", c->side, launch_consistency(k, bp, nf, out + f0 * px, c->side));
    }
    CUDA_TRY(c, cudaEventRecord(c->ev_rows, c->side));
    CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_rows, 0));
  } else {
    if (ka.sweep)
      TIMED(c, "agg_sweep", s, launch_agg_sweep(ka, c->b, n, s));
    else
      TIMED(c, "agg_lines", s, launch_agg_lines(ka, c->b, n, c->spill8, s));
    TIMED(c, "agg_rows_wta", s, launch_agg_rows(ka, c->b, n, c->spill8, s));
    TIMED(c, "consistency", s, launch_consistency(k, c->b, n, out, s));
  }
  c->computed = true;
  c->last_n = n;
  c->front_n = 0;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_compute_banded(sgmf_ctx *c, int n, const uint8_t *left, const uint8_t *right,
                                           const float *lidar, const int16_t *band_lo, int16_t *out) {
  if (!c) return SGMF_ERR_ARG;
  if (!out || !band_lo) return fail(c, SGMF_ERR_ARG, "sgmf_compute_banded: NULL pointer");
  if (c->k.subpixel) return fail(c, SGMF_ERR_PARAM, "sgmf_compute_banded: subpixel must be 0");
  sgmf_status st = sgmf_compute_front(c, n, left, right, lidar);
  if (st != SGMF_OK) return st;
  return sgmf_compute_banded_back(c, n, band_lo, out);
}

extern "C" int sgmf_band_width(const sgmf_ctx *c) { return c ? c->k.band : 0; }
