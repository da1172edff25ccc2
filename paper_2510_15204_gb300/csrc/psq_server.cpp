// Serving runtime: a request loop for integral jobs of different sizes arriving over time.
//
// Jobs are admitted as device memory and stream slots free up (first-fit allocation in a
// caller-provided device arena, FIFO order with backfilling: a waiting job that fits runs
// even when an earlier, larger one does not yet).  Admitted jobs run concurrently, each on its
// own stream: its tables go up, psq_compute runs, the requested matrices come back to the
// caller's host buffers, and an event marks completion.  A worker thread polls completions,
// returns memory and slots, and admits the next jobs.  Nothing here waits on the GPU without
// a bound: completion is detected by cudaEventQuery.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "psq_internal.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Request {
  uint64_t ticket = 0;
  psq_job* job = nullptr;
  unsigned mask = 0;
  double* h_out[5] = {};
  size_t out_bytes[5] = {};
  size_t ws_bytes = 0, need = 0, off = 0;
  int slot = -1;
  int state = 0;  // 0 queued, 1 running, 2 done
  psq_status status = PSQ_OK;
  std::string message;
  double t_submit = 0, t_start = 0, t_done = 0;
};

// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
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
  std::map<size_t, size_t> free_;
};

}  // namespace

struct psq_server {
  psq_context* ctx = nullptr;
  int device = 0;
  char* arena_base = nullptr;
  size_t arena_bytes = 0;
  std::unique_ptr<Arena> arena;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<int*> status_host;  // page-locked status word per slot
  std::vector<int> slot_free;
  std::deque<Request*> queue;
  std::vector<Request*> running;
  std::map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  std::string fatal;
};

namespace {

// Launches one admitted request on its slot's stream (called with the server lock held).
void launch(psq_server* S, Request* r) {
  cudaStream_t s = S->streams[r->slot];
  char* base = S->arena_base + r->off;
  double* d_out[5] = {};
  size_t o = align256(r->ws_bytes);
  for (int c = 0; c < 5; ++c) {
    if (!((r->mask >> c) & 1)) continue;
    d_out[c] = (double*)(base + o);
    o += align256(r->out_bytes[c]);
  }
  r->t_start = now_s();
  psq_status st = psq::compute_on(r->job, r->mask, base, r->ws_bytes, d_out, s, true);
  if (st == PSQ_OK) {
    for (int c = 0; c < 5 && st == PSQ_OK; ++c) {
      if (!((r->mask >> c) & 1)) continue;
      if (cudaMemcpyAsync(r->h_out[c], d_out[c], r->out_bytes[c], cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = psq::set_error(PSQ_ERR_CUDA, "device-to-host copy failed");
    }
  }
  if (st == PSQ_OK) {
    const size_t so = psq::status_offset(r->job, r->mask);
    *S->status_host[r->slot] = 0;
    if (cudaMemcpyAsync(S->status_host[r->slot], base + so, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = psq::set_error(PSQ_ERR_CUDA, "status copy failed");
  }
  if (st == PSQ_OK && cudaEventRecord(S->events[r->slot], s) != cudaSuccess)
    st = psq::set_error(PSQ_ERR_CUDA, "event record failed");
  r->state = 1;
  r->status = st;
  if (st != PSQ_OK) r->message = psq_last_error();
}

void worker_main(psq_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    bool progress = false;
    // completions
    for (size_t i = 0; i < S->running.size();) {
      Request* r = S->running[i];
      bool finished = r->status != PSQ_OK;
      if (!finished) {
        const cudaError_t q = cudaEventQuery(S->events[r->slot]);
        if (q == cudaSuccess) {
          finished = true;
          if (*S->status_host[r->slot]) {
            r->status = PSQ_ERR_TIMEOUT;
            r->message = "a bounded device wait expired";
          }
        } else if (q != cudaErrorNotReady) {
          finished = true;
          r->status = PSQ_ERR_CUDA;
          r->message = cudaGetErrorString(q);
        }
      }
      if (finished) {
        if (r->status != PSQ_OK) cudaStreamSynchronize(S->streams[r->slot]);
        r->t_done = now_s();
        r->state = 2;
        S->arena->release(r->off, r->need);
        S->slot_free.push_back(r->slot);
        S->running[i] = S->running.back();
        S->running.pop_back();
        progress = true;
        S->cv.notify_all();
      } else {
        ++i;
      }
    }
    // admissions: queue order, any waiting job that fits (backfilling)
    for (auto it = S->queue.begin(); it != S->queue.end() && !S->slot_free.empty();) {
      Request* r = *it;
      size_t off = 0;
      if (S->arena->alloc(r->need, &off)) {
        r->off = off;
        r->slot = S->slot_free.back();
        S->slot_free.pop_back();
        launch(S, r);
        S->running.push_back(r);
        it = S->queue.erase(it);
        progress = true;
      } else {
        ++it;
      }
    }
    if (!progress) S->cv.wait_for(lk, std::chrono::microseconds(S->running.empty() ? 2000 : 20));
  }
}

}  // namespace

extern "C" {

psq_status psq_server_create(psq_context* ctx, void* d_arena, size_t arena_bytes, int max_inflight,
                             psq_server** out) {
  if (!out) return psq::set_error(PSQ_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ctx || !d_arena || arena_bytes < 4096 || max_inflight < 1 || max_inflight > 64)
    return psq::set_error(PSQ_ERR_ARG, "server needs a context, an arena and 1..64 slots");
  if ((uintptr_t)d_arena % 256) return psq::set_error(PSQ_ERR_ARG, "arena must be 256-byte aligned");
  if (psq::context_device(ctx) < 0) return psq::set_error(PSQ_ERR_ARG, "the context has no device (planning only)");
  psq_server* S = new (std::nothrow) psq_server();
  if (!S) return psq::set_error(PSQ_ERR_OOM, "server allocation failed");
  S->ctx = ctx;
  S->device = psq::context_device(ctx);
  S->arena_base = (char*)d_arena;
  S->arena_bytes = arena_bytes;
  S->arena.reset(new Arena(arena_bytes));
  cudaSetDevice(S->device);
  for (int i = 0; i < max_inflight; ++i) {
    cudaStream_t s;
    cudaEvent_t e;
    int* h = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&h, sizeof(int)) != cudaSuccess) {
      delete S;
      return psq::set_error(PSQ_ERR_CUDA, "stream/event creation failed");
    }
    S->streams.push_back(s);
    S->events.push_back(e);
    S->status_host.push_back(h);
    S->slot_free.push_back(i);
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return PSQ_OK;
}

psq_status psq_server_submit(psq_server* S, psq_job* job, unsigned mask, double* h_out[5], uint64_t* ticket) {
  if (!S || !job || !h_out || !ticket) return psq::set_error(PSQ_ERR_ARG, "NULL argument");
  if (mask == 0 || (mask & ~31u)) return psq::set_error(PSQ_ERR_ARG, "bad class mask");
  size_t ws = 0;
  psq_status st = psq_job_workspace(job, mask, &ws);  // plans on the caller's thread
  if (st != PSQ_OK) return st;
  int nbf = 0, naux = 0;
  psq_job_sizes(job, &nbf, &naux);
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return psq::set_error(PSQ_ERR_OOM, "request allocation failed");
  r->job = job;
  r->mask = mask;
  r->ws_bytes = ws;
  r->need = align256(ws);
  for (int c = 0; c < 5; ++c) {
    if (!((mask >> c) & 1)) continue;
    if (!h_out[c]) return psq::set_error(PSQ_ERR_ARG, "host output is NULL");
    r->h_out[c] = h_out[c];
    const size_t n = c < 3 ? (size_t)nbf * nbf : (c == 3 ? (size_t)naux * naux : (size_t)naux * nbf * nbf);
    r->out_bytes[c] = n * sizeof(double);
    r->need += align256(r->out_bytes[c]);
  }
  if (r->need > S->arena_bytes) return psq::set_error(PSQ_ERR_OOM, "job needs more device memory than the arena");
  std::lock_guard<std::mutex> lk(S->mu);
  r->ticket = S->next_ticket++;
  r->t_submit = now_s();
  *ticket = r->ticket;
  S->queue.push_back(r.get());
  S->all[r->ticket] = std::move(r);
  S->cv.notify_all();
  return PSQ_OK;
}

psq_status psq_server_poll(psq_server* S, uint64_t ticket, int* done, double* latency_s) {
  if (!S || !done) return psq::set_error(PSQ_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return psq::set_error(PSQ_ERR_ARG, "unknown ticket");
  Request* r = it->second.get();
  *done = r->state == 2;
  if (latency_s) *latency_s = *done ? r->t_done - r->t_submit : now_s() - r->t_submit;
  if (*done && r->status != PSQ_OK) return psq::set_error(r->status, r->message.c_str());
  return PSQ_OK;
}

psq_status psq_server_wait(psq_server* S, uint64_t ticket, double timeout_s) {
  if (!S) return psq::set_error(PSQ_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return psq::set_error(PSQ_ERR_ARG, "unknown ticket");
  Request* r = it->second.get();
  const double t_end = now_s() + timeout_s;
  while (r->state != 2) {
    if (now_s() > t_end) return psq::set_error(PSQ_ERR_TIMEOUT, "request not finished in time");
    S->cv.wait_for(lk, std::chrono::milliseconds(1));
  }
  if (r->status != PSQ_OK) return psq::set_error(r->status, r->message.c_str());
  return PSQ_OK;
}

psq_status psq_server_destroy(psq_server* S) {
  if (!S) return PSQ_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  for (auto s : S->streams) cudaStreamSynchronize(s);
  for (auto s : S->streams) cudaStreamDestroy(s);
  for (auto e : S->events) cudaEventDestroy(e);
  for (auto h : S->status_host) cudaFreeHost(h);
  delete S;
  return PSQ_OK;
}

}  // extern "C"
