// sgmf_serve.cu -- a request loop for several cameras with continuous batching.
//
// Requests (one stereo pair + LiDAR map in host memory) arrive from any
// thread.  Cameras of equal shape share one queue.  A worker thread owns all
// CUDA work: whenever a batched context ("slot") of a shape is idle it takes
// every waiting request of that shape (up to the slot's capacity), copies
// them into the slot's resident device buffers, runs the pipeline once for
// the whole batch and copies the outputs back, all on the slot's own stream.
// Requests that arrive meanwhile wait for the next idle slot, so batches form
// continuously while earlier ones are still on the GPU, and slots of
// different shapes (or several of one shape) overlap on the device.  Slots
// are created on demand while the device bytes they need fit the budget
// given at creation (admission by device memory); a camera whose shape does
// not fit even one slot is refused.  A host callback on the slot's stream
// stamps the completion time; the worker then checks the slot's device error
// word and hands the requests to sgmf_server_poll.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sgmf.h"
#include "sgmf_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t tag = 0;
  int camera = -1;
  const uint8_t *left = nullptr, *right = nullptr;
  const float *lidar = nullptr;
  int16_t *out = nullptr;
  Clock::time_point t_submit{}, t_done{};
  int status = SGMF_OK;
};

enum SlotState { kIdle, kBusy, kLanded };

struct Slot {
  int shape = -1;
  int W = 0, H = 0;
  int cap = 0;
  sgmf_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  uint8_t *dl = nullptr, *dr = nullptr;
  float *dli = nullptr;
  int16_t *dout = nullptr;
  size_t bytes = 0;
  SlotState state = kIdle;          // written by the worker and the stream callback under the lock
  std::vector<Request> batch;
  Clock::time_point landed{};
  struct sgmf_server *srv = nullptr;
};

struct Shape {
  int W = 0, H = 0, D = 0;
  std::deque<Request> waiting;
  std::vector<int> slots;
  size_t slot_bytes = 0;            // device bytes one slot needs (known after the first)
};

}  // namespace

struct sgmf_server {
  int device = 0;
  sgmf_params prm{};
  size_t budget = 0, used = 0, peak = 0;
  int max_batch = 1, max_slots = 2;
  // deques: elements keep their addresses while other threads append
  std::deque<Shape> shapes;
  std::vector<int> cam_shape;
  std::deque<Slot *> slots;
  std::deque<Request> done;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t submitted = 0, completed = 0, batches = 0, batched_frames = 0;
  int largest_batch = 0, max_concurrent = 0;
};

using sgmf::set_noctx_error;

static sgmf_status sfail(sgmf_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_noctx_error(buf);
  return s;
}

static void free_slot(Slot *sl) {
  if (!sl) return;
  if (sl->stream) cudaStreamSynchronize(sl->stream);
  sgmf_destroy(sl->ctx);
  for (void *p : {(void *)sl->dl, (void *)sl->dr, (void *)sl->dli, (void *)sl->dout})
    if (p) cudaFree(p);
  if (sl->stream) cudaStreamDestroy(sl->stream);
  delete sl;
}

// a slot of shape si = (W, H, D) (device allocations, lock not held; the
// caller registers it)
static sgmf_status make_slot(sgmf_server *s, int si, int W, int H, int D, Slot **out) {
  Slot *sl = new (std::nothrow) Slot();
  if (!sl) return SGMF_ERR_OOM;
  sl->shape = si;
  sl->W = W;
  sl->H = H;
  sl->cap = s->max_batch;
  sl->srv = s;
  sgmf_status st = sgmf_create_batched(W, H, D, sl->cap, &sl->ctx);
  if (st == SGMF_OK) st = sgmf_set_params(sl->ctx, &s->prm);
  const size_t px = (size_t)W * H * sl->cap;
  if (st == SGMF_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sl->dl, px);
    if (e == cudaSuccess) e = cudaMalloc(&sl->dr, px);
    if (e == cudaSuccess) e = cudaMalloc(&sl->dli, px * 4);
    if (e == cudaSuccess) e = cudaMalloc(&sl->dout, px * 2);
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? SGMF_ERR_OOM : SGMF_ERR_CUDA;
  }
  if (st == SGMF_OK) st = sgmf_set_stream(sl->ctx, sl->stream);
  if (st != SGMF_OK) {
    free_slot(sl);
    return st;
  }
  sl->bytes = sgmf_device_bytes(sl->ctx) + px * 8;
  *out = sl;
  return SGMF_OK;
}

// stream callback after a batch's outputs have landed in host memory: no CUDA calls here
static void CUDART_CB on_landed(void *arg) {
  Slot *sl = static_cast<Slot *>(arg);
  sgmf_server *s = sl->srv;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    sl->state = kLanded;
    sl->landed = Clock::now();
  }
  s->cv_work.notify_all();
}

// enqueue one batch on an idle slot (worker thread, lock NOT held)
static sgmf_status dispatch(Slot *sl) {
  const size_t fpx = (size_t)sl->W * sl->H;
  const int n = (int)sl->batch.size();
  bool any_lidar = false;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const Request &r = sl->batch[i];
    e = cudaMemcpyAsync(sl->dl + i * fpx, r.left, fpx, cudaMemcpyHostToDevice, sl->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl->dr + i * fpx, r.right, fpx, cudaMemcpyHostToDevice, sl->stream);
    if (e != cudaSuccess) break;
    if (r.lidar) {
      any_lidar = true;
      e = cudaMemcpyAsync(sl->dli + i * fpx, r.lidar, fpx * 4, cudaMemcpyHostToDevice, sl->stream);
    } else {
      e = cudaMemsetAsync(sl->dli + i * fpx, 0, fpx * 4, sl->stream);   // no returns for this frame
    }
  }
  if (e != cudaSuccess) return SGMF_ERR_CUDA;
  sgmf_status st = sgmf_compute_batch(sl->ctx, n, sl->dl, sl->dr, any_lidar ? sl->dli : nullptr, sl->dout);
  if (st != SGMF_OK) return st;
  for (int i = 0; i < n && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(sl->batch[i].out, sl->dout + i * fpx, fpx * 2, cudaMemcpyDeviceToHost, sl->stream);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(sl->stream, on_landed, sl);
  return e == cudaSuccess ? SGMF_OK : SGMF_ERR_CUDA;
}

static void worker_loop(sgmf_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lock(s->mu);
  for (;;) {
    bool progress = false;
    // 1. retire landed batches: check the device error word, hand requests out
    for (size_t k = 0; k < s->slots.size(); ++k) {
      Slot *sl = s->slots[k];
      if (sl->state != kLanded) continue;
      const Clock::time_point t = sl->landed;
      std::vector<Request> b;
      b.swap(sl->batch);
      lock.unlock();
      const sgmf_status st = sgmf_sync(sl->ctx);   // the stream is idle: reads the error word
      lock.lock();
      for (Request &r : b) {
        r.t_done = t;
        r.status = st;
        s->done.push_back(r);
      }
      s->completed += b.size();
      sl->state = kIdle;
      progress = true;
      s->cv_done.notify_all();
    }
    // 2. give every shape's waiting requests to an idle slot (or a new one)
    for (size_t si = 0; si < s->shapes.size(); ++si) {
      Shape &sh = s->shapes[si];                    // stable: shapes is a deque
      while (!sh.waiting.empty()) {
        Slot *idle = nullptr;
        for (int k : sh.slots)
          if (s->slots[k]->state == kIdle) {
            idle = s->slots[k];
            break;
          }
        if (!idle && (int)sh.slots.size() < s->max_slots && s->used + sh.slot_bytes <= s->budget) {
          const int W = sh.W, H = sh.H, D = sh.D;
          lock.unlock();
          Slot *nsl = nullptr;
          const sgmf_status st = make_slot(s, (int)si, W, H, D, &nsl);
          lock.lock();
          if (st == SGMF_OK && s->used + nsl->bytes <= s->budget) {
            s->used += nsl->bytes;
            s->peak = std::max(s->peak, s->used);
            sh.slot_bytes = nsl->bytes;
            sh.slots.push_back((int)s->slots.size());
            s->slots.push_back(nsl);
            idle = nsl;
          } else if (st == SGMF_OK) {
            sh.slot_bytes = nsl->bytes;   // does not fit after all: wait for a slot to go idle
            lock.unlock();
            free_slot(nsl);
            lock.lock();
          } else {
            sh.slot_bytes = s->budget + 1;   // creation failed: use the slots there are
          }
        }
        if (!idle) break;
        const int n = std::min<int>(idle->cap, (int)sh.waiting.size());
        idle->batch.assign(sh.waiting.begin(), sh.waiting.begin() + n);
        sh.waiting.erase(sh.waiting.begin(), sh.waiting.begin() + n);
        idle->state = kBusy;
        s->batches += 1;
        s->batched_frames += n;
        s->largest_batch = std::max(s->largest_batch, n);
        int busy = 0;
        for (size_t k = 0; k < s->slots.size(); ++k) busy += s->slots[k]->state != kIdle;
        s->max_concurrent = std::max(s->max_concurrent, busy);
        lock.unlock();
        const sgmf_status st = dispatch(idle);
        if (st != SGMF_OK) cudaStreamSynchronize(idle->stream);   // let enqueued copies finish
        lock.lock();
        if (st != SGMF_OK) {
          // no completion callback was enqueued: fail the batch here
          for (Request &r : idle->batch) {
            r.t_done = Clock::now();
            r.status = st;
            s->done.push_back(r);
          }
          s->completed += idle->batch.size();
          idle->batch.clear();
          idle->state = kIdle;
          s->cv_done.notify_all();
        }
        progress = true;
      }
    }
    if (progress) continue;
    bool busy = false;
    for (size_t k = 0; k < s->slots.size(); ++k) busy |= s->slots[k]->state != kIdle;
    bool waiting = false;
    for (size_t si = 0; si < s->shapes.size(); ++si) waiting |= !s->shapes[si].waiting.empty();
    if (s->stop && !busy && !waiting) break;
    s->cv_work.wait_for(lock, std::chrono::milliseconds(50));
  }
}

extern "C" sgmf_status sgmf_server_create(const sgmf_params *p, size_t device_budget_bytes, int max_batch,
                                          int max_slots_per_shape, sgmf_server **out) {
  if (!out) return sfail(SGMF_ERR_ARG, "sgmf_server_create: out is NULL");
  *out = nullptr;
  if (max_batch < 1 || max_batch > 256 || max_slots_per_shape < 1 || max_slots_per_shape > 16)
    return sfail(SGMF_ERR_ARG, "sgmf_server_create: need 1 <= max_batch <= 256 and 1 <= slots per shape <= 16");
  sgmf_params prm;
  sgmf_default_params(&prm);
  if (p) {
    std::string why;
    if (sgmf::validate_params(*p, why) != SGMF_OK) return sfail(SGMF_ERR_PARAM, "sgmf_server_create: %s", why.c_str());
    prm = *p;
  }
  sgmf_server *s = new (std::nothrow) sgmf_server();
  if (!s) return sfail(SGMF_ERR_OOM, "sgmf_server_create: host allocation failed");
  cudaGetDevice(&s->device);
  s->prm = prm;
  s->budget = device_budget_bytes;
  s->max_batch = max_batch;
  s->max_slots = max_slots_per_shape;
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return SGMF_OK;
}

extern "C" int sgmf_server_add_camera(sgmf_server *s, int width, int height, int max_disp) {
  if (!s) return -(int)sfail(SGMF_ERR_ARG, "sgmf_server_add_camera: NULL server");
  std::unique_lock<std::mutex> lock(s->mu);
  int si = -1;
  for (int i = 0; i < (int)s->shapes.size(); ++i)
    if (s->shapes[i].W == width && s->shapes[i].H == height && s->shapes[i].D == max_disp) si = i;
  if (si < 0) {
    // admission: the first slot of a new shape must fit the remaining budget
    Shape sh;
    sh.W = width;
    sh.H = height;
    sh.D = max_disp;
    s->shapes.push_back(sh);
    si = (int)s->shapes.size() - 1;
    lock.unlock();
    Slot *sl = nullptr;
    const sgmf_status st = make_slot(s, si, width, height, max_disp, &sl);
    lock.lock();
    if (st != SGMF_OK || s->used + sl->bytes > s->budget) {
      const size_t need = st == SGMF_OK ? sl->bytes : 0;
      s->shapes.pop_back();
      lock.unlock();
      if (st == SGMF_OK) free_slot(sl);
      if (st != SGMF_OK) return -(int)sfail(st, "sgmf_server_add_camera: %s", sgmf_last_error(nullptr));
      return -(int)sfail(SGMF_ERR_OOM, "sgmf_server_add_camera: %dx%d D=%d needs %zu device bytes, %zu of %zu left",
                         width, height, max_disp, need, s->budget - s->used, s->budget);
    }
    s->used += sl->bytes;
    s->peak = std::max(s->peak, s->used);
    s->shapes[si].slot_bytes = sl->bytes;
    s->shapes[si].slots.push_back((int)s->slots.size());
    s->slots.push_back(sl);
  }
  s->cam_shape.push_back(si);
  return (int)s->cam_shape.size() - 1;
}

extern "C" sgmf_status sgmf_server_submit(sgmf_server *s, int camera, const uint8_t *left, const uint8_t *right,
                                          const float *lidar, int16_t *out, uint64_t tag) {
  if (!s || !left || !right || !out) return sfail(SGMF_ERR_ARG, "sgmf_server_submit: NULL argument");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (camera < 0 || camera >= (int)s->cam_shape.size())
      return sfail(SGMF_ERR_ARG, "sgmf_server_submit: unknown camera %d", camera);
    if (s->stop) return sfail(SGMF_ERR_ARG, "sgmf_server_submit: server is shutting down");
    Request r;
    r.tag = tag;
    r.camera = camera;
    r.left = left;
    r.right = right;
    r.lidar = lidar;
    r.out = out;
    r.t_submit = Clock::now();
    s->shapes[s->cam_shape[camera]].waiting.push_back(r);
    ++s->submitted;
  }
  s->cv_work.notify_all();
  return SGMF_OK;
}

extern "C" int sgmf_server_poll(sgmf_server *s, int wait_ms, uint64_t *tag, int *camera, int *status,
                                double *latency_ms) {
  if (!s) return -(int)SGMF_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  if (s->done.empty()) return 0;
  const Request r = s->done.front();
  s->done.pop_front();
  if (tag) *tag = r.tag;
  if (camera) *camera = r.camera;
  if (status) *status = r.status;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  return 1;
}

extern "C" sgmf_status sgmf_server_stats(sgmf_server *s, sgmf_server_counters *out) {
  if (!s || !out) return SGMF_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->batches = s->batches;
  out->batched_frames = s->batched_frames;
  out->largest_batch = s->largest_batch;
  out->max_concurrent_batches = s->max_concurrent;
  out->slots = (int)s->slots.size();
  out->device_bytes = s->used;
  out->peak_device_bytes = s->peak;
  out->budget_bytes = s->budget;
  return SGMF_OK;
}

extern "C" void sgmf_server_destroy(sgmf_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();   // the worker drains waiting and in-flight batches first
  for (Slot *sl : s->slots) free_slot(sl);
  delete s;
}
