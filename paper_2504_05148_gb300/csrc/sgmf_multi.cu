// sgmf_multi.cu -- mixed-size batches replayed as one CUDA graph.
//
// Frames of equal shape form a class.  A class is one batched context: each
// kernel of the pipeline processes all of the class's frames in one launch.
// The classes are independent, so the capture forks them onto their own
// streams and joins them again; the instantiated graph holds them as
// parallel branches and one cudaGraphLaunch replays the whole batch.  Inputs
// and outputs live in resident per-class buffers (frame-major, like a
// batched context expects), so the captured pointers never change.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "sgmf.h"
#include "sgmf_internal.cuh"

namespace {

struct MultiClass {
  sgmf_shape shape{};
  int nf = 0;                    // frames in the class
  sgmf_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint8_t *left = nullptr, *right = nullptr;
  float *lidar = nullptr;
  int16_t *out = nullptr;
};

}  // namespace

struct sgmf_multi {
  int device = 0;
  std::vector<MultiClass> cls;
  std::vector<std::pair<int, int>> where;   // frame -> (class, slot)
  cudaStream_t origin = nullptr;            // capture stream, default launch stream
  cudaStream_t last = nullptr;              // stream of the last launch
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t bytes = 0;
};

using sgmf::set_noctx_error;

static sgmf_status mfail(sgmf_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_noctx_error(buf);
  return s;
}

static void drop_graph(sgmf_multi *m) {
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  m->exec = nullptr;
  m->graph = nullptr;
}

extern "C" void sgmf_multi_destroy(sgmf_multi *m) {
  if (!m) return;
  if (m->last) cudaStreamSynchronize(m->last);
  drop_graph(m);
  for (MultiClass &c : m->cls) {
    if (c.stream) cudaStreamSynchronize(c.stream);
    sgmf_destroy(c.ctx);
    for (void *p : {(void *)c.left, (void *)c.right, (void *)c.lidar, (void *)c.out})
      if (p) cudaFree(p);
    if (c.done) cudaEventDestroy(c.done);
    if (c.stream) cudaStreamDestroy(c.stream);
  }
  if (m->fork) cudaEventDestroy(m->fork);
  if (m->origin) cudaStreamDestroy(m->origin);
  delete m;
}

extern "C" sgmf_status sgmf_multi_create(const sgmf_shape *shapes, int n, const sgmf_params *p, sgmf_multi **out) {
  if (!out || !shapes) return mfail(SGMF_ERR_ARG, "sgmf_multi_create: NULL argument");
  *out = nullptr;
  if (n < 1 || n > 4096) return mfail(SGMF_ERR_SHAPE, "sgmf_multi_create: need 1 <= n <= 4096 (got %d)", n);
  sgmf_multi *m = new (std::nothrow) sgmf_multi();
  if (!m) return mfail(SGMF_ERR_OOM, "sgmf_multi_create: host allocation failed");
  cudaGetDevice(&m->device);
  // classes in order of first appearance
  std::map<std::tuple<int, int, int>, int> index;
  for (int i = 0; i < n; ++i) {
    const sgmf_shape s = shapes[i];
    auto key = std::make_tuple(s.width, s.height, s.max_disp);
    auto it = index.find(key);
    int ci;
    if (it == index.end()) {
      ci = (int)m->cls.size();
      index[key] = ci;
      m->cls.emplace_back();
      m->cls.back().shape = s;
    } else {
      ci = it->second;
    }
    m->where.emplace_back(ci, m->cls[ci].nf++);
  }
  sgmf_status st = SGMF_OK;
  auto cuda = [&](cudaError_t e, const char *what) {
    if (st == SGMF_OK && e != cudaSuccess)
      st = mfail(e == cudaErrorMemoryAllocation ? SGMF_ERR_OOM : SGMF_ERR_CUDA, "sgmf_multi_create: %s: %s", what,
                 cudaGetErrorString(e));
  };
  cuda(cudaStreamCreateWithFlags(&m->origin, cudaStreamNonBlocking), "stream");
  cuda(cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming), "event");
  for (MultiClass &c : m->cls) {
    if (st != SGMF_OK) break;
    sgmf_status cs = sgmf_create_batched(c.shape.width, c.shape.height, c.shape.max_disp, c.nf, &c.ctx);
    if (cs != SGMF_OK) {
      st = mfail(cs, "sgmf_multi_create: class %dx%d D=%d: %s", c.shape.width, c.shape.height, c.shape.max_disp,
                 sgmf_last_error(nullptr));
      break;
    }
    if (p && (cs = sgmf_set_params(c.ctx, p)) != SGMF_OK) {
      st = mfail(cs, "sgmf_multi_create: %s", sgmf_last_error(c.ctx));
      break;
    }
    const size_t px = (size_t)c.shape.width * c.shape.height * c.nf;
    cuda(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "stream");
    cuda(cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming), "event");
    cuda(cudaMalloc(&c.left, px), "cudaMalloc");
    cuda(cudaMalloc(&c.right, px), "cudaMalloc");
    cuda(cudaMalloc(&c.lidar, px * 4), "cudaMalloc");
    cuda(cudaMalloc(&c.out, px * 2), "cudaMalloc");
    if (st == SGMF_OK) {
      cuda(cudaMemset(c.left, 0, px), "cudaMemset");
      cuda(cudaMemset(c.right, 0, px), "cudaMemset");
      cuda(cudaMemset(c.lidar, 0, px * 4), "cudaMemset");
      cuda(cudaMemset(c.out, 0xff, px * 2), "cudaMemset");
      cs = sgmf_set_stream(c.ctx, c.stream);
      m->bytes += px * 7 + sgmf_device_bytes(c.ctx);
    }
  }
  if (st != SGMF_OK) {
    sgmf_multi_destroy(m);
    return st;
  }
  *out = m;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_multi_frame(sgmf_multi *m, int i, uint8_t **left, uint8_t **right, float **lidar,
                                        int16_t **out) {
  if (!m) return mfail(SGMF_ERR_ARG, "sgmf_multi_frame: NULL batch");
  if (i < 0 || i >= (int)m->where.size())
    return mfail(SGMF_ERR_ARG, "sgmf_multi_frame: frame %d out of range [0, %zu)", i, m->where.size());
  const MultiClass &c = m->cls[m->where[i].first];
  const size_t off = (size_t)m->where[i].second * c.shape.width * c.shape.height;
  if (left) *left = c.left + off;
  if (right) *right = c.right + off;
  if (lidar) *lidar = c.lidar + off;
  if (out) *out = c.out + off;
  return SGMF_OK;
}

extern "C" int sgmf_multi_classes(const sgmf_multi *m) { return m ? (int)m->cls.size() : 0; }

extern "C" sgmf_status sgmf_multi_class_info(const sgmf_multi *m, int cls, sgmf_shape *shape, int *frames,
                                             sgmf_tuning *t) {
  if (!m || cls < 0 || cls >= (int)m->cls.size()) return mfail(SGMF_ERR_ARG, "sgmf_multi_class_info: bad class");
  const MultiClass &c = m->cls[cls];
  if (shape) *shape = c.shape;
  if (frames) *frames = c.nf;
  if (t) sgmf_get_tuning(c.ctx, t);
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_multi_autotune(sgmf_multi *m, int reps) {
  if (!m) return mfail(SGMF_ERR_ARG, "sgmf_multi_autotune: NULL batch");
  if (m->last) cudaStreamSynchronize(m->last);
  drop_graph(m);
  for (MultiClass &c : m->cls) {
    sgmf_status st = sgmf_autotune(c.ctx, c.nf, c.left, c.right, c.lidar, c.out, reps, nullptr, nullptr);
    if (st != SGMF_OK) return mfail(st, "sgmf_multi_autotune: %s", sgmf_last_error(c.ctx));
  }
  return SGMF_OK;
}

// every class once on its own stream, outside any capture: first-use kernel
// attributes are set here, not inside the capture
static sgmf_status run_classes(sgmf_multi *m) {
  for (MultiClass &c : m->cls) {
    sgmf_status st = sgmf_compute_batch(c.ctx, c.nf, c.left, c.right, c.lidar, c.out);
    if (st != SGMF_OK) return mfail(st, "sgmf_multi_launch: %s", sgmf_last_error(c.ctx));
  }
  for (MultiClass &c : m->cls) {
    sgmf_status st = sgmf_sync(c.ctx);
    if (st != SGMF_OK) return mfail(st, "sgmf_multi_launch: %s", sgmf_last_error(c.ctx));
  }
  return SGMF_OK;
}

static sgmf_status capture(sgmf_multi *m) {
  cudaError_t e = cudaStreamBeginCapture(m->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return mfail(SGMF_ERR_CUDA, "sgmf_multi_launch: begin capture: %s", cudaGetErrorString(e));
  sgmf_status st = SGMF_OK;
  e = cudaEventRecord(m->fork, m->origin);
  for (MultiClass &c : m->cls) {
    if (e != cudaSuccess || st != SGMF_OK) break;
    e = cudaStreamWaitEvent(c.stream, m->fork, 0);
    if (e != cudaSuccess) break;
    st = sgmf_compute_batch(c.ctx, c.nf, c.left, c.right, c.lidar, c.out);
    if (st != SGMF_OK) {
      st = mfail(st, "sgmf_multi_launch: capture: %s", sgmf_last_error(c.ctx));
      break;
    }
    e = cudaEventRecord(c.done, c.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->origin, c.done, 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(m->origin, &g);
  if (st != SGMF_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (st != SGMF_OK) return st;
    return mfail(SGMF_ERR_CUDA, "sgmf_multi_launch: capture: %s",
                 cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  m->graph = g;
  e = cudaGraphInstantiate(&m->exec, g, 0);
  if (e != cudaSuccess) {
    drop_graph(m);
    return mfail(SGMF_ERR_CUDA, "sgmf_multi_launch: instantiate: %s", cudaGetErrorString(e));
  }
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_multi_launch(sgmf_multi *m, void *stream) {
  if (!m) return mfail(SGMF_ERR_ARG, "sgmf_multi_launch: NULL batch");
  if (!m->exec) {
    sgmf_status st = run_classes(m);
    if (st == SGMF_OK) st = capture(m);
    if (st != SGMF_OK) return st;
  }
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : m->origin;
  const cudaError_t e = cudaGraphLaunch(m->exec, s);
  if (e != cudaSuccess) return mfail(SGMF_ERR_CUDA, "sgmf_multi_launch: cudaGraphLaunch: %s", cudaGetErrorString(e));
  m->last = s;
  return SGMF_OK;
}

extern "C" sgmf_status sgmf_multi_sync(sgmf_multi *m) {
  if (!m) return mfail(SGMF_ERR_ARG, "sgmf_multi_sync: NULL batch");
  if (m->last) {
    const cudaError_t e = cudaStreamSynchronize(m->last);
    if (e != cudaSuccess) return mfail(SGMF_ERR_CUDA, "sgmf_multi_sync: %s", cudaGetErrorString(e));
  }
  for (MultiClass &c : m->cls) {
    const sgmf_status st = sgmf_sync(c.ctx);   // reads the class's device error word
    if (st != SGMF_OK) return mfail(st, "sgmf_multi_sync: %s", sgmf_last_error(c.ctx));
  }
  return SGMF_OK;
}

extern "C" int sgmf_multi_launches(const sgmf_multi *m) {
  if (!m) return 0;
  int n = 0;
  for (const MultiClass &c : m->cls) n += sgmf_launches_per_compute(c.ctx);
  return n;
}

extern "C" size_t sgmf_multi_device_bytes(const sgmf_multi *m) { return m ? m->bytes : 0; }
