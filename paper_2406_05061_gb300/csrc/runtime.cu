// Host runtime around progot_solve: a batched solve over many independent problems and
// a continuous-batching server with a device-memory budget.
//
// Both run each problem through progot_solve on one of several CUDA streams, each
// driven by its own host thread: a problem's Sinkhorn loop reads its device state back
// once per chunk of iterations, so several problems in flight keep the GPU busy while
// one of them waits for its readback, and small problems (whose persistent sweeps use
// only part of the 152 SMs) run side by side. Every kernel's launch configuration
// depends only on its problem's sizes, so a result is bit-identical whether the problem
// runs alone or among others.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/progot.h"
#include "progot_internal.h"

namespace progot {

static size_t round_up256(size_t v) { return (v + 255) & ~size_t(255); }

static int check_problem(const progot_problem& p) {
  if (p.x == nullptr || p.y == nullptr || p.n <= 0 || p.m <= 0 || p.d <= 0 || p.K <= 0 || p.alpha == nullptr ||
      p.eps == nullptr || p.tau == nullptr || p.x_out == nullptr || p.g_all == nullptr)
    return PROGOT_ERR_INVALID_ARG;
  return PROGOT_OK;
}

// Per-worker workspace for the largest problem of a batch.
static size_t slice_bytes(const progot_problem* probs, int32_t count, int32_t precision) {
  int64_t n = 1, m = 1;
  int32_t d = 1;
  for (int i = 0; i < count; ++i) {
    n = std::max<int64_t>(n, probs[i].n);
    m = std::max<int64_t>(m, probs[i].m);
    d = std::max<int32_t>(d, probs[i].d);
  }
  return round_up256(progot_workspace_size(n, m, d, precision));
}

// Engine of progot_solve_batched: 1 = one persistent launch over the whole batch
// (batch_tc.cu) when every problem fits it, 0 = per-problem solves on host-driven streams.
static std::atomic<int> g_batch_engine{1};

static bool persistent_eligible(const progot_problem* probs, int32_t count, int32_t precision) {
  if (precision != PROGOT_BF16X3 && precision != PROGOT_BF16) return false;
  for (int i = 0; i < count; ++i)
    if (probs[i].d > 64 || probs[i].n > ((int64_t)1 << 24) || probs[i].m > ((int64_t)1 << 24)) return false;
  return true;
}

}  // namespace progot

using namespace progot;

extern "C" {

int progot_set_batch_engine(int32_t engine) {
  if (engine != 0 && engine != 1) {
    set_last_error_message("engine must be 0 (streams) or 1 (persistent)");
    return PROGOT_ERR_INVALID_ARG;
  }
  g_batch_engine.store(engine);
  return PROGOT_OK;
}

size_t progot_batched_workspace_size(const progot_problem* problems, int32_t count, int32_t precision,
                                     int32_t n_streams) {
  if (problems == nullptr || count <= 0 || n_streams <= 0) return 0;
  size_t need = slice_bytes(problems, count, precision) * (size_t)n_streams + 256;
  if (g_batch_engine.load() == 1 && persistent_eligible(problems, count, precision))
    need = std::max(need, progot_batch_plan_workspace_size(problems, count, precision));
  return need;
}

int progot_solve_batched(progot_problem* problems, int32_t count, int32_t max_iter, int32_t precision,
                         int32_t n_streams, void* workspace, size_t ws_bytes, progot_stream_t stream) {
  set_last_error_message("");
  if (problems == nullptr || count <= 0 || n_streams <= 0 || workspace == nullptr) {
    set_last_error_message("problems, count > 0, n_streams > 0 and a workspace are required");
    return PROGOT_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    if (check_problem(problems[i]) != PROGOT_OK) {
      set_last_error_message("a problem has a NULL pointer or a non-positive size");
      return PROGOT_ERR_INVALID_ARG;
    }
  }
  if (g_batch_engine.load() == 1 && persistent_eligible(problems, count, precision) &&
      ws_bytes >= progot_batch_plan_workspace_size(problems, count, precision)) {
    // one persistent launch over the whole batch
    progot_batch_plan* plan = nullptr;
    int rc = progot_batch_plan_create(problems, count, max_iter, precision, workspace, ws_bytes, &plan);
    if (rc) return rc;
    rc = progot_batch_plan_run(plan, 0, stream);
    if (!rc) rc = progot_batch_plan_collect(plan, problems, stream);
    progot_batch_plan_destroy(plan);
    return rc;
  }
  const size_t slice = slice_bytes(problems, count, precision);
  if (ws_bytes < slice * (size_t)n_streams) {
    set_last_error_message("batched workspace too small (see progot_batched_workspace_size)");
    return PROGOT_ERR_WORKSPACE;
  }
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(workspace) + 255) & ~uintptr_t(255));
  if (base + slice * (size_t)n_streams > reinterpret_cast<char*>(workspace) + ws_bytes) {
    set_last_error_message("batched workspace too small after 256-byte alignment");
    return PROGOT_ERR_WORKSPACE;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_last_error_message("cudaGetDevice failed");
    return PROGOT_ERR_CUDA;
  }
  // largest problems first (longest-processing-time order)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)problems[a].n * problems[a].m * problems[a].d > (double)problems[b].n * problems[b].m * problems[b].d;
  });
  cudaStream_t caller = (cudaStream_t)stream;
  cudaEvent_t start_ev = nullptr;
  if (cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(start_ev, caller) != cudaSuccess) {
    set_last_error_message("event creation failed");
    return PROGOT_ERR_CUDA;
  }
  std::atomic<int> next{0};
  std::vector<cudaStream_t> streams(n_streams, nullptr);
  std::vector<cudaEvent_t> done_ev(n_streams, nullptr);
  std::atomic<int> setup_fail{0};
  auto worker = [&](int w) {
    if (cudaSetDevice(dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done_ev[w], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamWaitEvent(streams[w], start_ev, 0) != cudaSuccess) {
      setup_fail = 1;
      return;
    }
    void* ws = base + slice * (size_t)w;
    for (;;) {
      const int j = next.fetch_add(1);
      if (j >= count) break;
      progot_problem& p = problems[order[j]];
      p.status = progot_solve(p.x, p.a, p.n, p.y, p.b, p.m, p.d, p.K, p.alpha, p.eps, p.tau, max_iter, precision,
                              p.x_out, p.g_all, p.f_last, nullptr, p.iters, p.errs, ws, slice, streams[w]);
    }
    cudaEventRecord(done_ev[w], streams[w]);
  };
  std::vector<std::thread> threads;
  threads.reserve(n_streams);
  for (int w = 0; w < n_streams; ++w) threads.emplace_back(worker, w);
  for (auto& t : threads) t.join();
  int rc = PROGOT_OK;
  for (int w = 0; w < n_streams; ++w) {
    if (done_ev[w]) cudaStreamWaitEvent(caller, done_ev[w], 0);
  }
  for (int w = 0; w < n_streams; ++w) {
    if (streams[w]) {
      cudaStreamSynchronize(streams[w]);
      cudaStreamDestroy(streams[w]);
    }
    if (done_ev[w]) cudaEventDestroy(done_ev[w]);
  }
  cudaEventDestroy(start_ev);
  if (setup_fail) {
    set_last_error_message("creating a worker stream or event failed");
    return PROGOT_ERR_CUDA;
  }
  for (int i = 0; i < count && rc == PROGOT_OK; ++i)
    if (problems[i].status != PROGOT_OK && problems[i].status != PROGOT_ERR_NOT_CONVERGED) rc = problems[i].status;
  if (rc == PROGOT_OK)
    for (int i = 0; i < count; ++i)
      if (problems[i].status == PROGOT_ERR_NOT_CONVERGED) rc = PROGOT_ERR_NOT_CONVERGED;
  if (rc == PROGOT_ERR_NOT_CONVERGED) set_last_error_message("at least one problem did not reach its tau");
  return rc;
}

}  // extern "C"

// ====================================================================== server
namespace progot {

// First-fit sub-allocator over one device arena (offsets, 256-byte granules).
class Arena {
 public:
  explicit Arena(size_t bytes) : size_(bytes) { free_[0] = bytes; }
  // returns the offset or SIZE_MAX
  size_t alloc(size_t bytes) {
    bytes = round_up256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, left = it->second - bytes;
        free_.erase(it);
        if (left) free_[off + bytes] = left;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }
  size_t size() const { return size_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

struct Request {
  progot_problem prob;  // host pointers
  std::chrono::steady_clock::time_point t_submit;
  double latency_ms = 0.0;
  int32_t status = PROGOT_OK;
  bool done = false;
  size_t bytes = 0;
};

}  // namespace progot

struct progot_server {
  int device = 0;
  int32_t precision = PROGOT_BF16X3;
  int32_t max_iter = 10000;
  char* arena_base = nullptr;
  progot::Arena* arena = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_mem, cv_done;
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, progot::Request> reqs;
  int64_t next_id = 0;
  int64_t completed = 0;
  int64_t in_flight = 0;
  bool stopping = false;
  std::vector<std::thread> workers;
};

namespace progot {

// Device bytes of one request: inputs, outputs and its solve workspace (each 256-aligned).
static size_t request_bytes(const progot_problem& p, int32_t precision) {
  const size_t f = sizeof(float);
  size_t b = 0;
  b += round_up256(f * (size_t)p.n * p.d) + round_up256(f * (size_t)p.m * p.d);             // x, y
  if (p.a) b += round_up256(f * (size_t)p.n);
  if (p.b) b += round_up256(f * (size_t)p.m);
  b += round_up256(f * (size_t)p.n * p.d) + round_up256(f * (size_t)p.K * p.m) + round_up256(f * (size_t)p.n);
  b += round_up256(progot_workspace_size(p.n, p.m, p.d, precision));
  return b;
}

static void serve(progot_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    size_t off = SIZE_MAX;
    Request* rq = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // admission: the head of the queue runs as soon as a worker is free and its
      // memory fits in the arena (first-fit); otherwise wait for a release
      for (;;) {
        if (S->stopping && S->queue.empty()) {
          lk.unlock();
          if (st) cudaStreamDestroy(st);
          return;
        }
        if (!S->queue.empty()) {
          rq = &S->reqs[S->queue.front()];
          off = S->arena->alloc(rq->bytes);
          if (off != SIZE_MAX) {
            S->queue.pop_front();
            S->in_flight += 1;
            break;
          }
          S->cv_mem.wait(lk);
        } else {
          S->cv_work.wait(lk);
        }
      }
    }
    // carve the request's device memory and run it
    const progot_problem& hp = rq->prob;
    char* base = S->arena_base + off;
    size_t o = 0;
    auto take = [&](size_t bytes) -> char* {
      char* q = base + o;
      o += round_up256(bytes);
      return q;
    };
    const size_t f = sizeof(float);
    float* x = (float*)take(f * hp.n * hp.d);
    float* y = (float*)take(f * hp.m * hp.d);
    float* a = hp.a ? (float*)take(f * hp.n) : nullptr;
    float* b = hp.b ? (float*)take(f * hp.m) : nullptr;
    float* x_out = (float*)take(f * hp.n * hp.d);
    float* g_all = (float*)take(f * hp.K * hp.m);
    float* f_last = (float*)take(f * hp.n);
    const size_t wsb = round_up256(progot_workspace_size(hp.n, hp.m, hp.d, S->precision));
    void* ws = take(wsb);
    int32_t rc = PROGOT_OK;
    if (cudaMemcpyAsync(x, hp.x, f * hp.n * hp.d, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(y, hp.y, f * hp.m * hp.d, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        (a && cudaMemcpyAsync(a, hp.a, f * hp.n, cudaMemcpyHostToDevice, st) != cudaSuccess) ||
        (b && cudaMemcpyAsync(b, hp.b, f * hp.m, cudaMemcpyHostToDevice, st) != cudaSuccess))
      rc = PROGOT_ERR_CUDA;
    if (rc == PROGOT_OK)
      rc = progot_solve(x, a, hp.n, y, b, hp.m, hp.d, hp.K, hp.alpha, hp.eps, hp.tau, S->max_iter, S->precision,
                        x_out, g_all, f_last, nullptr, hp.iters, hp.errs, ws, wsb, st);
    if (rc == PROGOT_OK || rc == PROGOT_ERR_NOT_CONVERGED) {
      if (cudaMemcpyAsync(hp.x_out, x_out, f * hp.n * hp.d, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(hp.g_all, g_all, f * hp.K * hp.m, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          (hp.f_last && cudaMemcpyAsync(hp.f_last, f_last, f * hp.n, cudaMemcpyDeviceToHost, st) != cudaSuccess))
        rc = PROGOT_ERR_CUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = PROGOT_ERR_CUDA;
    const auto t_end = std::chrono::steady_clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->arena->release(off, rq->bytes);
      rq->status = rc;
      rq->latency_ms = std::chrono::duration<double, std::milli>(t_end - rq->t_submit).count();
      rq->done = true;
      S->in_flight -= 1;
      S->completed += 1;
    }
    S->cv_mem.notify_all();
    S->cv_done.notify_all();
  }
}

}  // namespace progot

extern "C" {

progot_server* progot_server_create(size_t budget_bytes, int32_t n_workers, int32_t precision, int32_t max_iter) {
  set_last_error_message("");
  if (budget_bytes < 1024 || n_workers <= 0 || max_iter < 0 ||
      (precision != PROGOT_FP32 && precision != PROGOT_BF16X3 && precision != PROGOT_BF16)) {
    set_last_error_message("budget >= 1 KiB, n_workers > 0, max_iter >= 0 and a valid precision are required");
    return nullptr;
  }
  progot_server* S = new (std::nothrow) progot_server();
  if (S == nullptr) return nullptr;
  cudaGetDevice(&S->device);
  S->precision = precision;
  S->max_iter = max_iter;
  void* mem = nullptr;
  if (cudaMalloc(&mem, budget_bytes) != cudaSuccess) {
    set_last_error_message("cudaMalloc of the serving arena failed");
    delete S;
    return nullptr;
  }
  S->arena_base = (char*)mem;
  S->arena = new progot::Arena(budget_bytes);
  for (int w = 0; w < n_workers; ++w) S->workers.emplace_back(progot::serve, S);
  return S;
}

int64_t progot_server_submit(progot_server* S, const progot_problem* req) {
  if (S == nullptr || req == nullptr || progot::check_problem(*req) != PROGOT_OK) {
    set_last_error_message("invalid server or request");
    return -PROGOT_ERR_INVALID_ARG;
  }
  const size_t bytes = progot::request_bytes(*req, S->precision);
  if (bytes > S->arena->size()) {
    set_last_error_message("request needs more device memory than the server's budget");
    return -PROGOT_ERR_OOM;
  }
  int64_t id;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    id = S->next_id++;
    progot::Request& r = S->reqs[id];
    r.prob = *req;
    r.t_submit = std::chrono::steady_clock::now();
    r.bytes = bytes;
    S->queue.push_back(id);
  }
  S->cv_work.notify_one();
  S->cv_mem.notify_all();
  return id;
}

int progot_server_wait(progot_server* S, int64_t id, double* latency_ms) {
  if (S == nullptr) return PROGOT_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) {
    set_last_error_message("unknown request id");
    return PROGOT_ERR_INVALID_ARG;
  }
  S->cv_done.wait(lk, [&] { return it->second.done; });
  const int32_t status = it->second.status;
  if (latency_ms) *latency_ms = it->second.latency_ms;
  S->reqs.erase(it);
  return status;
}

int progot_server_stats(progot_server* S, int64_t* completed, int64_t* in_flight, size_t* bytes_in_use,
                        size_t* peak_bytes) {
  if (S == nullptr) return PROGOT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (completed) *completed = S->completed;
  if (in_flight) *in_flight = S->in_flight;
  if (bytes_in_use) *bytes_in_use = S->arena->used();
  if (peak_bytes) *peak_bytes = S->arena->peak();
  return PROGOT_OK;
}

void progot_server_destroy(progot_server* S) {
  if (S == nullptr) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  S->cv_mem.notify_all();
  for (auto& t : S->workers) t.join();
  cudaFree(S->arena_base);
  delete S->arena;
  delete S;
}

}  // extern "C"
