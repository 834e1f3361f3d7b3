// Render server (adop_serve_*): keeps point clouds resident, admits render
// requests of mixed resolution by memory, batches them into launches and
// overlaps batches on several CUDA streams (continuous batching: requests
// that arrive while others run are admitted as soon as a slot and memory
// free up and launched on the next free stream).
//
// Threads: the caller's threads submit / wait / poll; one scheduler thread
// admits, launches and reaps.  Completion of a batch is signalled by a host
// function enqueued on its stream (it only flips an atomic flag, stamps the
// time and notifies; it makes no CUDA call).  Every wait is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "launch.h"
#include "serve_core.h"

namespace adop {
namespace serve {
namespace {

using Clock = std::chrono::steady_clock;

adop_status err(adop_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
adop_status err(adop_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return st;
}

enum ReqState : int { kQueued = 0, kAdmitted = 1, kLaunched = 2, kDone = 3, kCancelled = 4, kFailed = 5 };

struct Request {
  uint64_t ticket = 0;
  int32_t cloud = 0;
  adop_camera cam{};
  void* out = nullptr;
  size_t bytes = 0;        // pixel state reserved in the pool
  size_t offset = SIZE_MAX;
  Clock::time_point t_submit;
  double latency_ms = 0.0;
  int state = kQueued;
  adop_status status = ADOP_OK;
};

struct Batch {
  std::vector<uint64_t> tickets;
  int stream = -1;
  std::atomic<bool> done{false};
  Clock::time_point t_done;
  std::condition_variable* cv = nullptr;
};

void CUDART_CB on_batch_done(void* p) {
  Batch* b = static_cast<Batch*>(p);
  b->t_done = Clock::now();
  b->done.store(true, std::memory_order_release);
  b->cv->notify_all();
}

size_t state_bytes(const adop_camera& cam, int levels, int c) {
  const int64_t px = pyramid_pixels(cam.K.w, cam.K.h, levels, nullptr);
  const size_t a = 256;
  auto up = [&](size_t v) { return (v + a - 1) / a * a; };
  return up((size_t)px * 8) + up((size_t)px * 4) + up((size_t)px * c * 4);
}

}  // namespace

struct Server {
  adop_serve_config cfg{};
  char* pool = nullptr;
  RangeAllocator alloc;
  std::vector<cudaStream_t> streams;
  std::vector<bool> stream_busy;
  std::vector<adop_points> clouds;
  int32_t c = 0;
  adop_dtype feat_dtype = ADOP_F32;

  std::mutex mu;
  std::condition_variable cv;       // scheduler wake-ups and batch completions
  std::condition_variable done_cv;  // request completions (waiters)
  AdmissionQueue<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<uint64_t> admitted;   // admitted, not yet launched
  std::vector<std::unique_ptr<Batch>> inflight;
  uint64_t next_ticket = 1;
  int active = 0;                   // admitted + launched requests (slots in use)
  bool stop = false;
  std::thread worker;

  // statistics
  LatencyStats lat;
  int64_t n_submitted = 0, n_completed = 0, n_cancelled = 0, n_failed = 0, n_batches = 0, n_batched_reqs = 0;
  int64_t n_mixed = 0;  // batches whose cameras render more than one cloud
  double points_done = 0.0;
  Clock::time_point t_start = Clock::now(), t_last{};
  bool any_done = false;

  void run();
  void reap_locked();
  void admit_locked();
  void launch_locked();
};

void Server::reap_locked() {
  for (size_t b = 0; b < inflight.size();) {
    Batch* bt = inflight[b].get();
    if (!bt->done.load(std::memory_order_acquire)) {
      ++b;
      continue;
    }
    for (uint64_t t : bt->tickets) {
      Request& r = reqs[t];
      alloc.release(r.offset);
      r.offset = SIZE_MAX;
      r.latency_ms = std::chrono::duration<double, std::milli>(bt->t_done - r.t_submit).count();
      r.state = kDone;
      lat.add(r.latency_ms);
      ++n_completed;
      points_done += (double)clouds[r.cloud].n;
      --active;
    }
    any_done = true;
    t_last = bt->t_done;
    stream_busy[bt->stream] = false;
    inflight.erase(inflight.begin() + b);
  }
}

void Server::admit_locked() {
  while (!queue.empty() && active < cfg.max_slots) {
    Request& r = reqs[queue.front()];
    const size_t off = alloc.alloc(r.bytes);
    if (off == SIZE_MAX) break;  // strict FIFO: the head waits for memory
    r.offset = off;
    r.state = kAdmitted;
    admitted.push_back(r.ticket);
    queue.pop();
    ++active;
  }
}

void Server::launch_locked() {
  while (!admitted.empty()) {
    int s = -1;
    for (size_t k = 0; k < streams.size(); ++k)
      if (!stream_busy[k]) {
        s = (int)k;
        break;
      }
    if (s < 0) return;
    // dynamic batching: a batch smaller than max_batch waits while its oldest
    // request is younger than the batching window (more requests may join)
    if ((int)admitted.size() < cfg.max_batch && cfg.batch_window_us > 0) {
      const double waited_us =
          std::chrono::duration<double, std::micro>(Clock::now() - reqs[admitted.front()].t_submit).count();
      if (waited_us < (double)cfg.batch_window_us) return;
    }
    // one batch: the oldest admitted requests, up to max_batch, of any cloud
    // (each camera of a launch renders its own cloud)
    const size_t take = std::min(admitted.size(), (size_t)cfg.max_batch);
    std::vector<uint64_t> pick(admitted.begin(), admitted.begin() + take);
    admitted.erase(admitted.begin(), admitted.begin() + take);

    LaunchCams lc;
    for (size_t j = 0; j < pick.size(); ++j) {
      Request& r = reqs[pick[j]];
      DevCam& d = lc.c[j];
      set_camera_constants(d, r.cam, cfg.levels, cfg.flags);
      const adop_points& P = clouds[r.cloud];
      d.xyz = P.xyz;
      d.feat = P.feat;
      d.normals = (cfg.flags & ADOP_FLAG_NORMAL_CULL) ? P.normals : nullptr;
      d.n = P.n;
      char* base = pool + r.offset;
      const int64_t px = d.off[cfg.levels];
      const size_t kb = (size_t)px * 8, cb = (size_t)px * 4;
      auto up = [](size_t v) { return (v + 255) / 256 * 256; };
      unsigned long long* key = reinterpret_cast<unsigned long long*>(base);
      uint32_t* cnt = reinterpret_cast<uint32_t*>(base + up(kb));
      d.acc = reinterpret_cast<float*>(base + up(kb) + up(cb));
      const size_t es = cfg.out_dtype == ADOP_F32 ? 4 : 2;
      char* img = static_cast<char*>(r.out);
      for (int l = 0; l < cfg.levels; ++l) {
        d.key[l] = key + d.off[l];
        d.cnt[l] = cnt + d.off[l];
        d.image[l] = img + (size_t)d.off[l] * c * es;
      }
      r.state = kLaunched;
    }
    PointArgs a{};  // (the point passes read each camera's cloud from its DevCam)
    a.background = cfg.background;
    a.env = cfg.env;
    a.env_w = cfg.env_w;
    a.env_h = cfg.env_h;
    a.radius = nullptr;
    a.beta = nullptr;
    a.levels = cfg.levels;
    a.ncam = (int32_t)pick.size();
    a.n = most_points(lc, a);
    a.znear = cfg.znear;
    a.a1 = 1.0f + cfg.alpha;
    a.flags = cfg.flags;
    cudaStream_t st = streams[s];
    const PdlScope pdl(pdl_for_points(a.n, a.ncam));
    cudaError_t e = launch_clear(lc, a, c, st);
    if (e == cudaSuccess) e = launch_depth(lc, a, st);
    if (e == cudaSuccess) e = launch_accum(lc, a, c, feat_dtype, st);
    if (e == cudaSuccess) e = launch_normalize(lc, a, c, cfg.out_dtype, st);
    if (e == cudaSuccess && cfg.env) e = launch_env_fill(lc, a, c, cfg.out_dtype, st);
    auto bt = std::make_unique<Batch>();
    bt->tickets = pick;
    bt->stream = s;
    bt->cv = &cv;
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_batch_done, bt.get());
    if (e != cudaSuccess) {
      for (uint64_t t : pick) {
        Request& r = reqs[t];
        alloc.release(r.offset);
        r.offset = SIZE_MAX;
        r.state = kFailed;
        r.status = ADOP_ERR_CUDA;
        ++n_failed;
        --active;
      }
      cudaGetLastError();
      done_cv.notify_all();
      continue;
    }
    stream_busy[s] = true;
    ++n_batches;
    n_batched_reqs += (int64_t)pick.size();
    for (uint64_t t : pick)
      if (reqs[t].cloud != reqs[pick.front()].cloud) {
        ++n_mixed;
        break;
      }
    inflight.push_back(std::move(bt));
  }
}

void Server::run() {
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    const size_t before = (size_t)n_completed;
    reap_locked();
    if ((size_t)n_completed != before) done_cv.notify_all();
    if (stop && queue.empty() && admitted.empty() && inflight.empty()) break;
    if (!stop) {
      admit_locked();
      launch_locked();
    } else {
      // on shutdown, queued requests are cancelled; admitted ones still run
      while (!queue.empty()) {
        Request& r = reqs[queue.front()];
        r.state = kCancelled;
        r.status = ADOP_ERR_CANCELLED;
        ++n_cancelled;
        queue.pop();
      }
      launch_locked();
      done_cv.notify_all();
    }
    // sleep until a submit, a completion or a short poll interval (which also
    // ends a batching window)
    cv.wait_for(lk, std::chrono::microseconds(cfg.batch_window_us > 0 && cfg.batch_window_us < 200
                                                  ? cfg.batch_window_us : 200));
  }
}

}  // namespace serve
}  // namespace adop

using adop::serve::Server;
using namespace adop::serve;

extern "C" {

adop_status adop_serve_create(const adop_serve_config* cfg, adop_server** out) {
  if (!cfg || !out) return err(ADOP_ERR_INVALID_ARG, "config and out must not be NULL");
  *out = nullptr;
  if (cfg->mem_budget_bytes < (1u << 20)) return err(ADOP_ERR_INVALID_ARG, "mem_budget_bytes below 1 MiB");
  if (cfg->max_slots < 1 || cfg->max_slots > 4096) return err(ADOP_ERR_INVALID_ARG, "max_slots outside [1, 4096]");
  if (cfg->streams < 1 || cfg->streams > 16) return err(ADOP_ERR_INVALID_ARG, "streams outside [1, 16]");
  if (cfg->max_batch < 1 || cfg->max_batch > adop::kMaxCamsPerLaunch)
    return err(ADOP_ERR_INVALID_ARG, "max_batch outside [1, %d]", adop::kMaxCamsPerLaunch);
  if (cfg->batch_window_us < 0 || cfg->batch_window_us > 1000000)
    return err(ADOP_ERR_INVALID_ARG, "batch_window_us outside [0, 10^6]");
  if (cfg->levels < 1 || cfg->levels > ADOP_MAX_LEVELS) return err(ADOP_ERR_INVALID_ARG, "levels outside [1, 8]");
  if (!(cfg->alpha >= 0.0f) || !(cfg->znear >= 0.0f)) return err(ADOP_ERR_INVALID_ARG, "alpha and znear must be >= 0");
  if (cfg->out_dtype != ADOP_F32 && cfg->out_dtype != ADOP_BF16 && cfg->out_dtype != ADOP_F16)
    return err(ADOP_ERR_INVALID_ARG, "unknown output dtype");
  if (cfg->flags & ~(uint32_t)(ADOP_FLAG_EPILOGUE | ADOP_FLAG_NORMAL_CULL))
    return err(ADOP_ERR_INVALID_ARG, "server flags may only be ADOP_FLAG_EPILOGUE | ADOP_FLAG_NORMAL_CULL");
  if (cfg->env && (!adop::env_size_ok(cfg->env_w, cfg->env_h) || ((uintptr_t)cfg->env & 15) != 0))
    return err(ADOP_ERR_INVALID_ARG, "environment map size outside [1, 16384]^2 or misaligned");
  auto s = std::make_unique<Server>();
  s->cfg = *cfg;
  cudaError_t e = cudaMalloc(&s->pool, cfg->mem_budget_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return err(ADOP_ERR_OUT_OF_MEMORY, "cudaMalloc of the %zu-byte budget: %s", cfg->mem_budget_bytes,
               cudaGetErrorString(e));
  }
  s->alloc = RangeAllocator(cfg->mem_budget_bytes, 256);
  s->streams.resize(cfg->streams);
  s->stream_busy.assign(cfg->streams, false);
  for (auto& st : s->streams) {
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
      for (auto& x : s->streams)
        if (x) cudaStreamDestroy(x);
      cudaFree(s->pool);
      return err(ADOP_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
  }
  Server* raw = s.release();
  raw->worker = std::thread([raw] { raw->run(); });
  *out = reinterpret_cast<adop_server*>(raw);
  return ADOP_OK;
}

adop_status adop_serve_load_cloud(adop_server* srv, const adop_points* pts, int32_t* cloud_id) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !pts || !cloud_id) return err(ADOP_ERR_INVALID_ARG, "server, points and cloud_id must not be NULL");
  if (pts->n < 1 || pts->n >= ((int64_t)1 << 31) || !pts->xyz || !pts->feat)
    return err(ADOP_ERR_INVALID_ARG, "cloud needs 1 <= n < 2^31 points and xyz/feat pointers");
  if (!adop::channels_supported(pts->c)) return err(ADOP_ERR_UNSUPPORTED, "channel count %d has no kernels", pts->c);
  if (((uintptr_t)pts->feat & 15) != 0) return err(ADOP_ERR_INVALID_ARG, "feat must be 16-byte aligned");
  if ((s->cfg.flags & ADOP_FLAG_NORMAL_CULL) && !pts->normals)
    return err(ADOP_ERR_INVALID_ARG, "normal culling needs normals");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->clouds.empty() && (pts->c != s->c || pts->feat_dtype != s->feat_dtype))
    return err(ADOP_ERR_INVALID_ARG, "all clouds of a server share one channel count and feature dtype");
  s->c = pts->c;
  s->feat_dtype = pts->feat_dtype;
  s->clouds.push_back(*pts);
  *cloud_id = (int32_t)s->clouds.size() - 1;
  return ADOP_OK;
}

adop_status adop_serve_submit(adop_server* srv, int32_t cloud_id, const adop_camera* cam, void* out_image,
                              uint64_t* ticket) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !cam || !out_image || !ticket) return err(ADOP_ERR_INVALID_ARG, "NULL argument");
  const adop_intrinsics& K = cam->K;
  if (K.w < 1 || K.h < 1 || K.w > 16384 || K.h > 16384 || (K.w >> (s->cfg.levels - 1)) < 1 ||
      (K.h >> (s->cfg.levels - 1)) < 1)
    return err(ADOP_ERR_INVALID_ARG, "image size %dx%d invalid for %d levels", K.w, K.h, s->cfg.levels);
  const float v[21] = {K.fx, K.fy, K.cx, K.cy, K.k1, K.k2, K.k3, K.p1, K.p2, cam->T.R[0], cam->T.R[1],
                       cam->T.R[2], cam->T.R[3], cam->T.R[4], cam->T.R[5], cam->T.R[6], cam->T.R[7], cam->T.R[8],
                       cam->T.t[0], cam->T.t[1], cam->T.t[2]};
  for (float x : v)
    if (!std::isfinite(x)) return err(ADOP_ERR_INVALID_ARG, "non-finite camera parameter");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return err(ADOP_ERR_CANCELLED, "server is shutting down");
  if (cloud_id < 0 || cloud_id >= (int32_t)s->clouds.size()) return err(ADOP_ERR_INVALID_ARG, "unknown cloud %d", cloud_id);
  Request r;
  r.ticket = s->next_ticket++;
  r.cloud = cloud_id;
  r.cam = *cam;
  r.out = out_image;
  r.bytes = state_bytes(*cam, s->cfg.levels, s->c);
  if (s->alloc.round(r.bytes) > s->alloc.capacity())
    return err(ADOP_ERR_OUT_OF_MEMORY, "request needs %zu bytes of pixel state, the budget is %zu", r.bytes,
               s->alloc.capacity());
  r.t_submit = Clock::now();
  *ticket = r.ticket;
  s->queue.push(r.ticket);
  s->reqs.emplace(r.ticket, r);
  ++s->n_submitted;
  s->cv.notify_all();
  return ADOP_OK;
}

adop_status adop_serve_poll(adop_server* srv, uint64_t ticket) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return err(ADOP_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return err(ADOP_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  switch (it->second.state) {
    case kDone: return ADOP_OK;
    case kCancelled: return err(ADOP_ERR_CANCELLED, "request %llu was cancelled", (unsigned long long)ticket);
    case kFailed: return err(it->second.status, "request %llu failed", (unsigned long long)ticket);
    default: return ADOP_ERR_BUSY;
  }
}

adop_status adop_serve_wait(adop_server* srv, uint64_t ticket, int32_t timeout_ms) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return err(ADOP_ERR_INVALID_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return err(ADOP_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (it->second.state < kDone) {
    if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state < kDone)
      return err(ADOP_ERR_TIMEOUT, "request %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
  }
  if (it->second.state == kDone) return ADOP_OK;
  if (it->second.state == kCancelled) return err(ADOP_ERR_CANCELLED, "request was cancelled");
  return err(it->second.status, "request failed");
}

adop_status adop_serve_cancel(adop_server* srv, uint64_t ticket) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return err(ADOP_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return err(ADOP_ERR_INVALID_ARG, "unknown ticket");
  if (it->second.state != kQueued) return ADOP_ERR_BUSY;  // already admitted: it runs to completion
  s->queue.remove_if_first([&](uint64_t t) { return t == ticket; });
  it->second.state = kCancelled;
  it->second.status = ADOP_ERR_CANCELLED;
  ++s->n_cancelled;
  s->done_cv.notify_all();
  return ADOP_OK;
}

adop_status adop_serve_latency(adop_server* srv, uint64_t ticket, double* ms) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !ms) return err(ADOP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return err(ADOP_ERR_INVALID_ARG, "unknown ticket");
  if (it->second.state != kDone) return ADOP_ERR_BUSY;
  *ms = it->second.latency_ms;
  return ADOP_OK;
}

adop_status adop_serve_get_stats(adop_server* srv, adop_serve_stats* st) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s || !st) return err(ADOP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof(*st));
  st->submitted = s->n_submitted;
  st->completed = s->n_completed;
  st->cancelled = s->n_cancelled;
  st->failed = s->n_failed;
  st->queued = (int64_t)s->queue.size();
  st->active = s->active;
  st->batches = s->n_batches;
  st->mean_batch = s->n_batches ? (double)s->n_batched_reqs / (double)s->n_batches : 0.0;
  st->p50_ms = s->lat.percentile(50.0);
  st->p99_ms = s->lat.percentile(99.0);
  st->mean_ms = s->lat.mean();
  st->max_ms = s->lat.max();
  const double span = s->any_done ? std::chrono::duration<double>(s->t_last - s->t_start).count() : 0.0;
  st->req_per_s = span > 0 ? (double)s->n_completed / span : 0.0;
  st->points_per_s = span > 0 ? s->points_done / span : 0.0;
  st->mem_in_use = s->alloc.in_use();
  st->mem_peak = s->alloc.peak();
  st->mixed_batches = s->n_mixed;
  return ADOP_OK;
}

adop_status adop_serve_reset_stats(adop_server* srv) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return err(ADOP_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->lat.clear();
  s->n_completed = s->n_batches = s->n_batched_reqs = s->n_mixed = 0;
  s->points_done = 0.0;
  s->any_done = false;
  s->t_start = Clock::now();
  return ADOP_OK;
}

adop_status adop_serve_destroy(adop_server* srv) {
  Server* s = reinterpret_cast<Server*>(srv);
  if (!s) return ADOP_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->worker.join();
  for (auto& st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(s->pool);
  delete s;
  return ADOP_OK;
}

}  // extern "C"
