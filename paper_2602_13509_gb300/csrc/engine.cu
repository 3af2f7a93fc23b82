// Serving engine: many concurrent sensor streams on one device with continuous batching.
//
// The paper processes one sensor (Sec. 3.1: one cube per core, pipelined) and proposes a
// line-based detector (Sec. 6.1). Serving generalises that to many streams sharing one
// GPU: each admitted stream is an hsad context (device-resident running statistics and
// factor, its own CUDA stream, so the work of different streams overlaps on the device);
// callers submit lines at any time; one worker thread repeatedly takes every stream's
// pending lines and pushes them as one batch (lines that arrived while the stream's
// previous batch was on the GPU form the next batch). Each stream replays a captured CUDA
// graph per batch size for the launches after its batch's first line (HSAD_CUDA_GRAPHS).
// Opening a stream with a new band count first runs the factor autotuner for it
// (hsad_autotune_factor). Admission is by the device-wide byte budget: a stream is opened
// only when its device memory fits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/hsad.h"

// internal helper of hsad_api.cu: 1 when every line of [first, first+n) has been scored,
// 0 while pending, negative on error
int hsadi_lines_ready(hsad_ctx* ctx, uint64_t first, int64_t n);
// internal helper of hsad_api.cu: 1 when a host push would not wait for a staging buffer
int hsadi_push_ready(hsad_ctx* ctx);

namespace {

using Clock = std::chrono::steady_clock;

struct EStream {
  hsad_ctx* ctx = nullptr;
  int64_t line_bytes = 0;
  int64_t max_batch = 256;
  std::mutex ctx_mu;                 // serialises calls on ctx (worker push vs callers)
  std::mutex q_mu;                   // guards the queue and counters below
  std::deque<std::vector<uint8_t>> q;
  uint64_t submitted = 0;            // lines accepted by hsad_engine_submit
  uint64_t pushed = 0;               // lines handed to the device
  std::condition_variable pushed_cv;
  bool open = true;
};

}  // namespace

struct hsad_engine {
  int device = 0;
  std::mutex mu;                      // guards streams vector
  std::vector<std::shared_ptr<EStream>> streams;
  std::mutex wake_mu;
  std::condition_variable wake;
  std::atomic<bool> stop{false};
  std::atomic<int64_t> n_pushes{0}, n_lines{0}, max_batch_seen{0};
  std::atomic<int> last_error{0};
  std::thread worker;
};

namespace {

void worker_loop(hsad_engine* e) {
  std::vector<uint8_t> buf;
  cudaSetDevice(e->device);
  while (!e->stop.load()) {
    bool did = false;
    std::vector<std::shared_ptr<EStream>> snap;
    {
      std::lock_guard<std::mutex> g(e->mu);
      snap = e->streams;
    }
    for (auto& sp : snap) {
      if (!sp) continue;
      EStream& s = *sp;
      int64_t n = 0;
      {
        // a stream whose staging buffers are both in flight keeps its lines queued (they
        // join its next, larger batch) instead of holding up every other stream
        std::lock_guard<std::mutex> g(s.ctx_mu);
        if (!s.ctx || !hsadi_push_ready(s.ctx)) continue;
      }
      {
        std::lock_guard<std::mutex> g(s.q_mu);
        if (!s.open || s.q.empty()) continue;
        buf.clear();
        while (!s.q.empty()) {
          auto& front = s.q.front();
          const int64_t k = (int64_t)front.size() / s.line_bytes;
          if (n > 0 && n + k > s.max_batch) break;
          buf.insert(buf.end(), front.begin(), front.end());
          n += k;
          s.q.pop_front();
        }
      }
      if (n == 0) continue;
      int rc;
      {
        std::lock_guard<std::mutex> g(s.ctx_mu);
        uint64_t first = 0;
        rc = hsad_push_lines(s.ctx, buf.data(), n, HSAD_HOST, &first);
      }
      if (rc != HSAD_OK) e->last_error.store(rc);
      {
        std::lock_guard<std::mutex> g(s.q_mu);
        s.pushed += (uint64_t)n;
      }
      s.pushed_cv.notify_all();
      e->n_pushes.fetch_add(1);
      e->n_lines.fetch_add(n);
      int64_t m = e->max_batch_seen.load();
      while (n > m && !e->max_batch_seen.compare_exchange_weak(m, n)) {
      }
      did = true;
    }
    if (!did) {
      std::unique_lock<std::mutex> lk(e->wake_mu);
      e->wake.wait_for(lk, std::chrono::microseconds(200));
    }
  }
}

std::shared_ptr<EStream> get_stream(hsad_engine* e, int32_t id) {
  std::lock_guard<std::mutex> g(e->mu);
  if (id < 0 || id >= (int32_t)e->streams.size()) return nullptr;
  return e->streams[id];
}

}  // namespace

extern "C" {

int hsad_engine_create(int32_t device, int64_t budget_bytes, hsad_engine** out) {
  if (!out || budget_bytes < 0) return HSAD_E_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ndev <= 0 ? HSAD_E_CUDA : HSAD_E_INVALID;
  }
  hsad_set_device_budget(device, budget_bytes);
  hsad_engine* e = new hsad_engine();
  e->device = device;
  e->worker = std::thread(worker_loop, e);
  *out = e;
  return HSAD_OK;
}

int hsad_engine_open(hsad_engine* e, const hsad_config* cfg, int32_t* stream_id) {
  if (!e || !cfg || !stream_id) return HSAD_E_INVALID;
  hsad_config c = *cfg;
  c.device = e->device;
  c.flags |= HSAD_CUDA_GRAPHS;  // repeated small batches: replay captured launch sequences
  // measured factor launch shapes for this band count (kept per process; fast when known)
  const int32_t tune_lines = cfg->max_batch_lines > 0 ? std::min<int32_t>(cfg->max_batch_lines, 64) : 64;
  hsad_autotune_factor(e->device, cfg->bands, cfg->precision, tune_lines, nullptr, nullptr);
  hsad_ctx* ctx = nullptr;
  const int rc = hsad_create(&c, &ctx);
  if (rc != HSAD_OK) return rc;
  auto s = std::make_shared<EStream>();
  s->ctx = ctx;
  // bytes of one submitted line: raw lines when the stream has the front end
  s->line_bytes = (int64_t)cfg->width * (cfg->raw_bands > 0 ? cfg->raw_bands : cfg->bands) *
                  (cfg->in_dtype == HSAD_U16 ? 2 : 4);
  s->max_batch = cfg->max_batch_lines > 0 ? cfg->max_batch_lines : 256;
  std::lock_guard<std::mutex> g(e->mu);
  e->streams.push_back(s);
  *stream_id = (int32_t)e->streams.size() - 1;
  return HSAD_OK;
}

int hsad_engine_submit(hsad_engine* e, int32_t stream_id, const void* lines, int64_t n_lines,
                       uint64_t* first_line_id) {
  if (!e || !lines || n_lines <= 0) return HSAD_E_INVALID;
  auto s = get_stream(e, stream_id);
  if (!s) return HSAD_E_INVALID;
  {
    std::lock_guard<std::mutex> g(s->q_mu);
    if (!s->open) return HSAD_E_INVALID;
    if (first_line_id) *first_line_id = s->submitted;
    const uint8_t* p = (const uint8_t*)lines;
    s->q.emplace_back(p, p + n_lines * s->line_bytes);
    s->submitted += (uint64_t)n_lines;
  }
  e->wake.notify_one();
  return HSAD_OK;
}

int hsad_engine_results(hsad_engine* e, int32_t stream_id, uint64_t first_line_id, int64_t n_lines,
                        float* scores, uint8_t* mask, int32_t timeout_ms) {
  if (!e || n_lines <= 0) return HSAD_E_INVALID;
  auto s = get_stream(e, stream_id);
  if (!s) return HSAD_E_INVALID;
  const auto t0 = Clock::now();
  auto expired = [&]() {
    return timeout_ms >= 0 &&
           std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() >= timeout_ms;
  };
  {
    std::unique_lock<std::mutex> lk(s->q_mu);
    if (first_line_id + (uint64_t)n_lines > s->submitted) return HSAD_E_INVALID;
    while (s->pushed < first_line_id + (uint64_t)n_lines) {
      if (expired()) return HSAD_E_TIMEOUT;
      s->pushed_cv.wait_for(lk, std::chrono::microseconds(200));
    }
  }
  for (;;) {
    {
      std::lock_guard<std::mutex> g(s->ctx_mu);
      const int r = hsadi_lines_ready(s->ctx, first_line_id, n_lines);
      if (r < 0) return r;
      if (r == 1) return hsad_scores(s->ctx, first_line_id, n_lines, scores, mask, HSAD_HOST, -1);
    }
    if (expired()) return HSAD_E_TIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int hsad_engine_close(hsad_engine* e, int32_t stream_id) {
  if (!e) return HSAD_E_INVALID;
  std::shared_ptr<EStream> s;
  {
    std::lock_guard<std::mutex> g(e->mu);
    if (stream_id < 0 || stream_id >= (int32_t)e->streams.size() || !e->streams[stream_id]) return HSAD_E_INVALID;
    s = e->streams[stream_id];
    e->streams[stream_id].reset();
  }
  {
    std::lock_guard<std::mutex> g(s->q_mu);
    s->open = false;
  }
  std::lock_guard<std::mutex> g(s->ctx_mu);
  const int rc = hsad_destroy(s->ctx);  // waits (bounded) for in-flight work, frees its budget
  s->ctx = nullptr;
  return rc;
}

int hsad_engine_counters(hsad_engine* e, int64_t* lines, int64_t* pushes, int64_t* max_batch) {
  if (!e) return HSAD_E_INVALID;
  if (lines) *lines = e->n_lines.load();
  if (pushes) *pushes = e->n_pushes.load();
  if (max_batch) *max_batch = e->max_batch_seen.load();
  return e->last_error.load();
}

int hsad_engine_destroy(hsad_engine* e) {
  if (!e) return HSAD_OK;
  e->stop.store(true);
  e->wake.notify_all();
  if (e->worker.joinable()) e->worker.join();
  std::vector<std::shared_ptr<EStream>> all;
  {
    std::lock_guard<std::mutex> g(e->mu);
    all = e->streams;
  }
  for (auto& s : all)
    if (s && s->ctx) hsad_destroy(s->ctx);
  delete e;
  return HSAD_OK;
}

}  // extern "C"
