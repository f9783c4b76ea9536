// Request server: continuous batching of matvec requests over resident plans.
//
// Requests (plan, nrhs host densities) arrive from any host thread.  One
// dispatcher thread admits them onto a fixed set of streams: it takes the
// oldest pending request, adds every other pending request on the same plan
// (oldest first) while the right-hand sides fit a per-apply cap, and runs the
// group as one apply with their right-hand sides side by side.  A group is
// admitted only when a stream is free and its device footprint (staging
// buffers + the apply's workspace) fits in the server's memory arena, one
// device allocation of the byte budget made at creation; nothing is
// allocated while serving.  Requests that arrive while others run are
// admitted as streams and memory free up, so their work overlaps on the
// device.  A host function queued on the stream after the result copies
// marks the group's requests done and records their latency.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.h"
#include "dfmm.h"
#include "internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// bytes of one density or potential value: complex64, or complex128 for an FP64 plan
size_t elem_bytes(const dfmm_stats& st) { return st.arith == 64 ? 16 : 8; }

struct Request {
  int64_t ticket = 0;
  dfmm_plan_t plan = nullptr;
  const void* f_host = nullptr;
  void* u_host = nullptr;
  int nrhs = 0;
  double t_submit = 0, t_done = 0;
  int status = 1;   // 1 while pending or running, then a dfmm_status
};

// First-fit allocator over the arena [0, size).
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
  }
  // offset of a free range of n bytes, or -1
  int64_t alloc(size_t n) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[off + n] = len - n;
      return (int64_t)off;
    }
    return -1;
  }
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;   // offset -> length
};

}  // namespace

struct dfmm_server_s;

namespace {

struct Slot {
  dfmm_server_s* srv = nullptr;
  int index = 0;
  cudaStream_t stream = nullptr;
  bool busy = false;
  std::vector<std::shared_ptr<Request>> group;
  size_t off = 0, bytes = 0;   // arena range held by the running group
};

void CUDART_CB on_group_done(void* p);

}  // namespace

struct dfmm_server_s {
  int device = 0;
  size_t budget = 0;
  int max_rhs = 16;
  char* base = nullptr;                 // the arena's device memory
  Arena arena;
  std::vector<std::unique_ptr<Slot>> slots;
  std::mutex mu;
  std::condition_variable cv;           // dispatcher: new work, a finished group, stop
  std::condition_variable cv_done;      // waiters: a finished group
  std::deque<std::shared_ptr<Request>> pending;
  std::unordered_map<int64_t, std::shared_ptr<Request>> live;   // submitted, not yet collected
  int64_t next_ticket = 1;
  bool stop = false;
  int fail_next = 0;                    // testing aid: status the next group fails with (0 = none)
  std::thread worker;
  std::map<std::pair<int64_t, int>, size_t> ws_bytes;       // workspace bytes per (plan id, nrhs)
  // statistics
  int64_t n_done = 0, n_failed = 0, n_applies = 0, rhs_done = 0, points_rhs_done = 0;
  int running = 0, max_running = 0;
  double t_first_submit = 0, t_last_done = 0;
  std::vector<double> lat_ms;

  size_t footprint(dfmm_plan_t plan, int nrhs) {
    dfmm_stats st{};
    dfmm_plan_stats(plan, &st);
    // keyed by the plan's id: a destroyed plan's handle may come back for another plan
    auto key = std::make_pair(st.plan_id, nrhs);
    auto it = ws_bytes.find(key);
    if (it == ws_bytes.end()) {
      const int64_t w = dfmm_apply_workspace_bytes(plan, nrhs);
      it = ws_bytes.emplace(key, (size_t)std::max<int64_t>(w, 0)).first;
    }
    return 2 * align256((size_t)st.N * nrhs * elem_bytes(st)) + align256(it->second) + 256;
  }

  void finish(Slot& sl, int status) {   // under mu
    const double t = now_s();
    for (auto& r : sl.group) {
      r->t_done = t;
      r->status = status;
      dfmm::plan_release(r->plan);
      if (status == DFMM_OK) {
        ++n_done;
        rhs_done += r->nrhs;
        dfmm_stats st{};
        dfmm_plan_stats(r->plan, &st);
        points_rhs_done += st.N * r->nrhs;
        lat_ms.push_back(1e3 * (t - r->t_submit));
      } else {
        ++n_failed;
      }
    }
    if (status == DFMM_OK) ++n_applies;
    t_last_done = t;
    arena.release(sl.off, sl.bytes);
    sl.group.clear();
    sl.busy = false;
    --running;
    cv.notify_all();
    cv_done.notify_all();
  }

  // Starts a group on a free slot (mu not held).  Copies the densities in,
  // runs the apply inside the group's arena range, copies the results out and
  // queues the completion callback.
  void launch(Slot& sl, int total_rhs, int injected) {
    dfmm_plan_t plan = sl.group.front()->plan;
    dfmm_stats st{};
    dfmm_plan_stats(plan, &st);
    const size_t N = (size_t)st.N;
    const size_t eb = elem_bytes(st);
    char* p = base + sl.off;
    char* f_dev = p;
    char* u_dev = p + align256(N * total_rhs * eb);
    char* scratch = p + 2 * align256(N * total_rhs * eb);
    const size_t scratch_bytes = sl.bytes - 2 * align256(N * total_rhs * eb);
    int rc = injected;   // a failure injected on the host: nothing is queued for this group
    size_t k = 0;
    for (auto& r : sl.group) {
      if (rc != DFMM_OK) break;
      if (cudaMemcpyAsync(f_dev + k * N * eb, r->f_host, N * r->nrhs * eb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        rc = DFMM_ERR_CUDA;
      k += r->nrhs;
    }
    if (rc == DFMM_OK) rc = dfmm::apply_with_scratch(plan, f_dev, u_dev, total_rhs, sl.stream, scratch, scratch_bytes);
    if (rc == DFMM_OK) {
      k = 0;
      for (auto& r : sl.group) {
        if (cudaMemcpyAsync(r->u_host, u_dev + k * N * eb, N * r->nrhs * eb, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
          rc = DFMM_ERR_CUDA;
        k += r->nrhs;
      }
    }
    if (rc == DFMM_OK && cudaLaunchHostFunc(sl.stream, on_group_done, &sl) != cudaSuccess) rc = DFMM_ERR_CUDA;
    if (rc != DFMM_OK) {
      cudaStreamSynchronize(sl.stream);   // let whatever was queued finish before the range is reused
      std::lock_guard<std::mutex> g(mu);
      finish(sl, rc);
    }
  }

  void run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      bool progressed = true;
      while (progressed && !pending.empty()) {
        progressed = false;
        Slot* sl = nullptr;
        for (auto& s : slots)
          if (!s->busy) { sl = s.get(); break; }
        if (!sl) break;
        // the oldest request's plan, with every pending request on it that fits
        dfmm_plan_t plan = pending.front()->plan;
        std::vector<std::shared_ptr<Request>> group;
        int total = 0;
        for (auto& r : pending)
          if (r->plan == plan && (group.empty() || total + r->nrhs <= max_rhs)) {
            group.push_back(r);
            total += r->nrhs;
          }
        const size_t need = footprint(plan, total);
        if (need > budget) {   // can never run: fail the oldest request alone
          auto r = pending.front();
          pending.pop_front();
          r->status = DFMM_ERR_OOM;
          r->t_done = now_s();
          dfmm::plan_release(r->plan);
          ++n_failed;
          cv_done.notify_all();
          progressed = true;
          continue;
        }
        const int64_t off = arena.alloc(need);
        if (off < 0) break;   // wait for a running group to free memory
        for (auto& r : group) pending.erase(std::find(pending.begin(), pending.end(), r));
        sl->busy = true;
        sl->group = std::move(group);
        sl->off = (size_t)off;
        sl->bytes = need;
        max_running = std::max(max_running, ++running);
        const int injected = fail_next;
        fail_next = 0;
        lk.unlock();
        try {
          launch(*sl, total, injected);
        } catch (...) {   // a host-side failure while queueing: the group fails, the server goes on
          cudaStreamSynchronize(sl->stream);
          std::lock_guard<std::mutex> g(mu);
          if (sl->busy) finish(*sl, DFMM_ERR_INVALID);
        }
        lk.lock();
        progressed = true;
      }
      if (stop && pending.empty() && running == 0) break;
      cv.wait(lk);
    }
  }
};

namespace {

void CUDART_CB on_group_done(void* p) {
  Slot* sl = (Slot*)p;
  std::lock_guard<std::mutex> g(sl->srv->mu);
  sl->srv->finish(*sl, DFMM_OK);
}

int serr(int code, const char* msg) { return dfmm::set_error(code, msg); }

}  // namespace

extern "C" {

int dfmm_server_create(int streams, int64_t budget_bytes, int max_rhs, dfmm_server_t* out) {
  if (!out) return serr(DFMM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (streams < 1 || streams > 64) return serr(DFMM_ERR_INVALID, "streams must be in [1, 64]");
  if (budget_bytes < 1) return serr(DFMM_ERR_INVALID, "budget_bytes must be positive");
  if (max_rhs < 1 || max_rhs > 64) return serr(DFMM_ERR_INVALID, "max_rhs must be in [1, 64]");
  std::unique_ptr<dfmm_server_s> S(new dfmm_server_s());
  if (cudaGetDevice(&S->device) != cudaSuccess) return serr(DFMM_ERR_CUDA, "no current device");
  S->budget = (size_t)budget_bytes;
  S->max_rhs = max_rhs;
  if (cudaMalloc(&S->base, S->budget) != cudaSuccess) {
    cudaGetLastError();
    return serr(DFMM_ERR_OOM, "the server's memory arena could not be allocated");
  }
  S->arena.reset(S->budget);
  for (int i = 0; i < streams; ++i) {
    std::unique_ptr<Slot> sl(new Slot());
    sl->srv = S.get();
    sl->index = i;
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& x : S->slots) cudaStreamDestroy(x->stream);
      cudaFree(S->base);
      return serr(DFMM_ERR_CUDA, "stream creation failed");
    }
    S->slots.push_back(std::move(sl));
  }
  dfmm_server_s* raw = S.get();
  S->worker = std::thread([raw] { raw->run(); });
  *out = S.release();
  return DFMM_OK;
}

int dfmm_server_submit(dfmm_server_t s, dfmm_plan_t plan, const void* f_host, void* u_host, int nrhs, int64_t* ticket) {
  if (!s || !plan || !f_host || !u_host || !ticket) return serr(DFMM_ERR_INVALID, "null argument");
  if (nrhs < 1 || nrhs > 64) return serr(DFMM_ERR_INVALID, "nrhs must be in [1, 64]");
  if (!dfmm::plan_acquire(plan)) return serr(DFMM_ERR_INVALID, "not a live plan (never created, or destroyed)");
  auto r = std::make_shared<Request>();
  r->plan = plan;
  r->f_host = f_host;
  r->u_host = u_host;
  r->nrhs = nrhs;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) {
      dfmm::plan_release(plan);
      return serr(DFMM_ERR_INVALID, "the server is shutting down");
    }
    r->ticket = s->next_ticket++;
    if (s->t_first_submit == 0) s->t_first_submit = r->t_submit;
    s->pending.push_back(r);
    s->live[r->ticket] = r;
    *ticket = r->ticket;
  }
  s->cv.notify_all();
  return DFMM_OK;
}

int dfmm_server_wait(dfmm_server_t s, int64_t ticket, double timeout_seconds, double* latency_ms) {
  if (!s) return serr(DFMM_ERR_INVALID, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) return serr(DFMM_ERR_INVALID, "unknown or already collected ticket");
  std::shared_ptr<Request> r = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(0.0, timeout_seconds));
  while (r->status == 1) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->status == 1)
      return serr(DFMM_ERR_TIMEOUT, "the request has not finished yet");
  }
  s->live.erase(ticket);
  if (latency_ms) *latency_ms = 1e3 * (r->t_done - r->t_submit);
  if (r->status != DFMM_OK)
    return serr(r->status, r->status == DFMM_ERR_OOM         ? "the request does not fit in the server's memory budget"
                           : r->status == DFMM_ERR_CANCELLED ? "the request was cancelled"
                                                             : "the request's apply failed");
  return DFMM_OK;
}

int dfmm_server_cancel(dfmm_server_t s, int64_t ticket) {
  if (!s) return serr(DFMM_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->live.find(ticket);
  if (it == s->live.end()) return serr(DFMM_ERR_INVALID, "unknown or already collected ticket");
  auto q = std::find(s->pending.begin(), s->pending.end(), it->second);
  if (q == s->pending.end())
    return serr(DFMM_ERR_INVALID, it->second->status == 1 ? "the request has started; it will complete"
                                                          : "the request has finished");
  std::shared_ptr<Request> r = *q;
  s->pending.erase(q);
  r->status = DFMM_ERR_CANCELLED;
  r->t_done = now_s();
  dfmm::plan_release(r->plan);
  ++s->n_failed;
  s->cv_done.notify_all();
  return DFMM_OK;
}

int dfmm_server_fail_next(dfmm_server_t s, int status) {
  if (!s) return serr(DFMM_ERR_INVALID, "null server");
  if (status >= 0) return serr(DFMM_ERR_INVALID, "status must be a negative dfmm_status");
  std::lock_guard<std::mutex> g(s->mu);
  s->fail_next = status;
  return DFMM_OK;
}

int dfmm_server_stats(dfmm_server_t s, dfmm_server_report* out) {
  if (!s || !out) return serr(DFMM_ERR_INVALID, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  dfmm_server_report o{};
  o.requests_done = s->n_done;
  o.requests_failed = s->n_failed;
  o.applies = s->n_applies;
  o.rhs_done = s->rhs_done;
  o.points_rhs_done = s->points_rhs_done;
  o.max_concurrent_applies = s->max_running;
  o.pending = (int64_t)s->pending.size();
  o.wall_seconds = s->t_last_done > s->t_first_submit ? s->t_last_done - s->t_first_submit : 0.0;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    o.latency_p50_ms = v[v.size() / 2];
    o.latency_p99_ms = v[std::min(v.size() - 1, (size_t)(0.99 * v.size()))];
  }
  *out = o;
  return DFMM_OK;
}

int dfmm_server_destroy(dfmm_server_t s) {
  if (!s) return DFMM_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& sl : s->slots) {
    cudaStreamSynchronize(sl->stream);
    cudaStreamDestroy(sl->stream);
  }
  cudaFree(s->base);
  delete s;
  return DFMM_OK;
}

}  // extern "C"
