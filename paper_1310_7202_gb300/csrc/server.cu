// Serving form: a request loop around rlu_factor (declared in include/rlu_server.h).
//
// One worker thread owns the scheduling state. Each admitted request gets a slot (a CUDA
// stream of its own) and a block of the workspace arena; its Algorithm 1 pipeline is
// enqueued on that stream with rlu_factor, followed by a host function that stamps the
// completion time and hands the request back to the worker, which then frees its slot and
// arena block and admits whatever fits next. Requests on different slots run concurrently
// on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "../../include/rlu_server.h"

namespace rlu {
int32_t validate(const void* A, int32_t dtype, int64_t m, int64_t n, int64_t lda, int32_t k,
                 int32_t l, int32_t prec, const int32_t* P, const int32_t* Q, const void* L,
                 int64_t ldl, const void* U, int64_t ldu);
}

namespace {

constexpr int kMaxBypass = 64;
constexpr size_t kGranule = 256;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// First-fit allocator over [0, cap) in 256-byte granules; freed blocks coalesce.
class Arena {
 public:
  explicit Arena(size_t cap) { free_[0] = cap / kGranule * kGranule; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = std::max<size_t>(kGranule, (bytes + kGranule - 1) / kGranule * kGranule);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t start = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[start + bytes] = rest;
      used_[start] = bytes;
      in_use_ += bytes;
      peak_ = std::max(peak_, in_use_);
      *off = start;
      return true;
    }
    return false;
  }
  void release(size_t off) {
    auto u = used_.find(off);
    if (u == used_.end()) return;
    const size_t bytes = u->second;
    used_.erase(u);
    in_use_ -= bytes;
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
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;  // offset -> bytes
  std::map<size_t, size_t> used_;
  size_t in_use_ = 0, peak_ = 0;
};

struct Req {
  rlu_request r{};
  size_t ws = 0, off = 0;
  int slot = -1;
  int32_t state = RLU_REQ_QUEUED, status = RLU_OK;
  int64_t t_submit = 0, t_start = 0, t_done = 0;
  int bypassed = 0;  // times a later request was admitted while this one waited
};

struct DoneArg {
  rlu_server* s;
  int64_t id;
};

}  // namespace

struct rlu_server {
  int dev = 0;
  char* base = nullptr;
  size_t budget = 0;
  Arena* arena = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<int64_t> slot_req;  // request on each slot, -1 when free
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req> reqs;  // by id; a deque keeps references stable as it grows
  std::deque<int64_t> queue;
  std::vector<int64_t> completed;  // stamped by the host function, retired by the worker
  bool stop = false;
  int running = 0;
  int64_t n_done = 0, n_failed = 0, peak_running = 0, n_bypass = 0;
  std::thread worker;
};

namespace {

void CUDART_CB on_done(void* p) {
  DoneArg* a = static_cast<DoneArg*>(p);
  rlu_server* s = a->s;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->reqs[(size_t)a->id].t_done = now_ns();
    s->completed.push_back(a->id);
  }
  s->cv.notify_all();
  delete a;
}

void retire(rlu_server* s, Req& q, int32_t state, int32_t status) {
  q.state = state;
  q.status = status;
  s->arena->release(q.off);
  s->slot_req[(size_t)q.slot] = -1;
  --s->running;
  if (state == RLU_REQ_DONE) ++s->n_done;
  else ++s->n_failed;
}

// Picks requests to start (caller holds the lock): arrival order, a request that does not
// fit may be passed, but not more than kMaxBypass times.
std::vector<int64_t> admit(rlu_server* s) {
  std::vector<int64_t> start;
  std::vector<int64_t> waiting;  // earlier requests that did not fit in this scan
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    int slot = -1;
    for (size_t i = 0; i < s->slot_req.size(); ++i)
      if (s->slot_req[i] < 0) {
        slot = (int)i;
        break;
      }
    if (slot < 0) break;
    Req& q = s->reqs[(size_t)*it];
    size_t off = 0;
    if (s->arena->alloc(q.ws, &off)) {
      q.off = off;
      q.slot = slot;
      q.state = RLU_REQ_RUNNING;
      s->slot_req[(size_t)slot] = *it;
      ++s->running;
      s->peak_running = std::max<int64_t>(s->peak_running, s->running);
      if (!waiting.empty()) ++s->n_bypass;
      for (int64_t w : waiting) ++s->reqs[(size_t)w].bypassed;
      start.push_back(*it);
      it = s->queue.erase(it);
      continue;
    }
    if (q.bypassed >= kMaxBypass) break;  // it waits for memory; nothing passes it now
    waiting.push_back(*it);
    ++it;
  }
  return start;
}

void worker_main(rlu_server* s) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    for (int64_t id : s->completed) retire(s, s->reqs[(size_t)id], RLU_REQ_DONE, RLU_OK);
    s->completed.clear();
    std::vector<int64_t> start = admit(s);
    if (!start.empty()) {
      // enqueue outside the lock; the state of these requests is already RUNNING
      std::vector<Req*> rs;
      for (int64_t id : start) rs.push_back(&s->reqs[(size_t)id]);
      lk.unlock();
      std::vector<int32_t> st(start.size(), RLU_OK);
      std::vector<int64_t> t0(start.size(), 0);
      for (size_t i = 0; i < start.size(); ++i) {
        // fields read here were fixed at submission and admission (under the lock)
        const Req& q = *rs[i];
        const rlu_request& r = q.r;
        cudaStream_t stream = s->streams[(size_t)q.slot];
        t0[i] = now_ns();
        st[i] = rlu_factor(r.A, r.dtype, r.m, r.n, r.lda, r.k, r.l, r.seed, r.prec, r.P, r.Q,
                           r.L, r.ldl, r.U, r.ldu, r.info, s->base + q.off, q.ws, stream);
        if (st[i] == RLU_OK) {
          DoneArg* a = new DoneArg{s, start[i]};
          if (cudaLaunchHostFunc(stream, on_done, a) != cudaSuccess) {
            delete a;
            cudaGetLastError();
            st[i] = RLU_ECUDA;
          }
        }
        // a failed launch may have enqueued part of its work: drain it before the arena
        // block is handed to another request
        if (st[i] != RLU_OK) cudaStreamSynchronize(stream);
      }
      lk.lock();
      for (size_t i = 0; i < start.size(); ++i) {
        rs[i]->t_start = t0[i];
        if (st[i] != RLU_OK) retire(s, *rs[i], RLU_REQ_FAILED, st[i]);
      }
      s->cv.notify_all();
      continue;
    }
    if (s->stop && s->queue.empty() && s->running == 0) break;
    s->cv.notify_all();
    // sleep until a request completes, or one arrives while a slot is free, or shutdown;
    // a waiting request that did not fit is retried only after a completion
    const size_t queued = s->queue.size();
    s->cv.wait(lk, [s, queued] {
      return !s->completed.empty() || s->stop ||
             (s->queue.size() > queued && s->running < (int)s->slot_req.size());
    });
  }
}

}  // namespace

extern "C" int32_t rlu_server_create(size_t budget_bytes, int32_t max_inflight,
                                     rlu_server** out) {
  if (!out || budget_bytes < kGranule || max_inflight < 1 || max_inflight > 64)
    return RLU_EINVAL;
  *out = nullptr;
  rlu_server* s = new rlu_server();
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return RLU_ECUDA;
  }
  if (cudaMalloc(reinterpret_cast<void**>(&s->base), budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return RLU_ENOMEM;
  }
  s->arena = new Arena(budget_bytes);
  s->budget = budget_bytes;
  s->streams.resize((size_t)max_inflight);
  s->slot_req.assign((size_t)max_inflight, -1);
  for (auto& st : s->streams) {
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (auto& t : s->streams)
        if (t) cudaStreamDestroy(t);
      cudaFree(s->base);
      delete s->arena;
      delete s;
      return RLU_ECUDA;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return RLU_OK;
}

extern "C" int32_t rlu_server_submit(rlu_server* s, const rlu_request* r, int64_t* id) {
  if (!s || !r || !id) return RLU_EINVAL;
  RLU_TRY(rlu::validate(r->A, r->dtype, r->m, r->n, r->lda, r->k, r->l, r->prec, r->P, r->Q,
                        r->L, r->ldl, r->U, r->ldu));
  const size_t ws = rlu_workspace_size(r->m, r->n, r->k, r->l, r->prec);
  if (ws == 0) return RLU_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return RLU_EINVAL;
    // a request larger than the whole arena could never start
    if ((ws + kGranule - 1) / kGranule * kGranule > s->budget / kGranule * kGranule)
      return RLU_ENOMEM;
    Req q;
    q.r = *r;
    q.ws = ws;
    q.t_submit = now_ns();
    *id = (int64_t)s->reqs.size();
    s->reqs.push_back(q);
    s->queue.push_back(*id);
  }
  s->cv.notify_all();
  return RLU_OK;
}

extern "C" int32_t rlu_server_poll(rlu_server* s, int64_t id, int32_t* state, int32_t* status,
                                   int64_t* t_submit_ns, int64_t* t_start_ns,
                                   int64_t* t_done_ns) {
  if (!s) return RLU_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (id < 0 || id >= (int64_t)s->reqs.size()) return RLU_EINVAL;
  const Req& q = s->reqs[(size_t)id];
  if (state) *state = q.state;
  if (status) *status = q.status;
  if (t_submit_ns) *t_submit_ns = q.t_submit;
  if (t_start_ns) *t_start_ns = q.t_start;
  if (t_done_ns) *t_done_ns = q.state == RLU_REQ_DONE ? q.t_done : 0;
  return RLU_OK;
}

extern "C" int32_t rlu_server_wait_all(rlu_server* s) {
  if (!s) return RLU_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait(lk, [s] { return s->queue.empty() && s->running == 0 && s->completed.empty(); });
  return RLU_OK;
}

extern "C" int32_t rlu_server_stats(rlu_server* s, int64_t* out6) {
  if (!s || !out6) return RLU_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  out6[0] = (int64_t)s->reqs.size();
  out6[1] = s->n_done;
  out6[2] = s->n_failed;
  out6[3] = (int64_t)s->arena->peak();
  out6[4] = s->peak_running;
  out6[5] = s->n_bypass;
  return RLU_OK;
}

extern "C" int32_t rlu_server_destroy(rlu_server* s) {
  if (!s) return RLU_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  cudaFree(s->base);
  delete s->arena;
  delete s;
  return RLU_OK;
}
