// server.cu -- continuous batching of isprime requests.
//
// A request is a host array (h_in, n) and a host output (h_out).  submit()
// admits it and returns a ticket at once.  A dispatcher thread forms
// micro-batches from the requests that have arrived, as device memory (a
// fixed arena of the given budget) and one of several stream slots become
// free, and runs each batch as: copy-in, one batched launch (batched.cu)
// over all its arrays, copy-out, event.  Short requests (at most the
// context's serve_short_max elements) are batched apart from long ones and keep a
// slot of their own, so their latency is that of a one-launch warp batch on a
// high-priority stream; when their buffers are pinned host memory the kernel
// reads and writes them in place, with no copies.  Batches on different slots overlap
// on the device; a request that arrives while others run joins the next
// batch instead of waiting for the GPU to drain.  A completion thread polls
// the slots' events, frees their memory, wakes waiters and records each
// request's latency (completion - arrival).  The context's resident sieve is
// shared read-only by every batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace ip {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  const uint64_t* h_in = nullptr;
  uint8_t* h_out = nullptr;
  size_t n = 0;
  Clock::time_point arrival;
  size_t off = 0;  // arena offset of the device copy (in bytes)
  size_t bytes = 0;
  // Short requests whose buffers are pinned host memory are read and written
  // by the kernel in place (through their device mappings): no arena, no copies.
  bool direct = false;
  const uint64_t* d_in = nullptr;
  uint8_t* d_out = nullptr;
  bool done = false;
  int status = ISPRIME_OK;
};
using RequestP = std::shared_ptr<Request>;

// First-fit allocator over [0, size) with coalescing; 256-byte granules.
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t next = it->first + bytes;
        free_.erase(it);
        if (rest) free_[next] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
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

 private:
  std::map<size_t, size_t> free_;
};

struct Slot {
  cudaStream_t stream = nullptr;  // long batches
  cudaStream_t fast = nullptr;    // short batches: the device's highest stream priority, so
                                  // their blocks are scheduled ahead of pending long work
  cudaEvent_t done_ev = nullptr;
  BatchState bs;
  std::vector<RequestP> reqs;
  bool busy = false;
};

}  // namespace
}  // namespace ip

struct isprime_server {
  isprime_ctx* ctx = nullptr;
  size_t budget = 0;
  char* d_arena = nullptr;
  std::unique_ptr<ip::Arena> arena;
  std::vector<ip::Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work;  // dispatcher: new requests, freed slots or memory
  std::condition_variable cv_done;  // waiters: requests completed
  std::condition_variable cv_comp;  // completer: batches in flight
  std::deque<ip::RequestP> pending;
  std::unordered_map<uint64_t, ip::RequestP> tickets;
  std::deque<int> inflight;
  bool stopping = false;
  uint64_t next_ticket = 1;
  std::thread dispatcher, completer;
  size_t small_cut = 0;  // requests of at most this many elements form short batches
  size_t long_cut = (size_t)1 << 24;  // a long batch grows to at most this many elements
  int fatal = ISPRIME_OK;
  std::string fatal_msg;
  // statistics
  std::vector<double> latency_ms;
  std::vector<uint8_t> latency_short;  // 1 where latency_ms[i] is a short request's
  uint64_t requests = 0, elements = 0, batches = 0;
  ip::Clock::time_point first_arrival, last_done;
  bool any = false;
};

namespace ip {
namespace {

constexpr size_t kMaxBatchRequests = 4096;
// A long batch stops growing at 2^serve_long_log2 elements (after its first
// request; the context's tuning), so that batches in flight stay short enough
// to overlap and rotate.

size_t request_bytes(size_t n) { return ((8 * n + 255) & ~(size_t)255) + ((n + 255) & ~(size_t)255); }

void fail_batch(Slot& sl, int st) {
  for (auto& r : sl.reqs) {
    r->status = st;
    r->done = true;
  }
}

// Size classes.  A request of at most small_cut elements (the context's
// serve_short_max) is "short": short requests are batched only with each
// other, up to small_cut elements per batch, which run as one-launch warp
// batches; the last slot
// never takes a batch of long requests, so a short request never waits for a
// long batch to finish.  Within a class requests keep their arrival order.
bool is_short(const isprime_server* S, const Request& r) { return r.n <= S->small_cut; }

// The device address of pinned (page-locked, mapped) host memory, if h is such memory.
bool device_view(const void* h, void** d) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA-known pointer: clear the error
    return false;
  }
  // only the unified-addressing case, where the device uses the host address itself
  if (a.type != cudaMemoryTypeHost || a.devicePointer != h) return false;
  *d = a.devicePointer;
  return true;
}

// A free slot for a batch of the class, or -1.
int free_slot(const isprime_server* S, bool short_class) {
  const size_t ns = S->slots.size();
  const size_t usable = (short_class || ns == 1 || S->small_cut == 0) ? ns : ns - 1;
  for (size_t i = 0; i < usable; ++i)
    if (!S->slots[i].busy) return (int)i;
  return -1;
}

// The class to serve next (that of the oldest pending request that has a
// free slot), or -1 if nothing pending can start now.
int next_class(const isprime_server* S, int* slot) {
  bool seen[2] = {false, false};
  for (const RequestP& r : S->pending) {
    const int c = is_short(S, *r) ? 1 : 0;
    if (seen[c]) continue;
    seen[c] = true;
    const int sl = free_slot(S, c == 1);
    if (sl >= 0) {
      *slot = sl;
      return c;
    }
    if (seen[0] && seen[1]) break;
  }
  return -1;
}

void dispatcher_loop(isprime_server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // wait for work that has a free slot of its class
    int slot = -1, cls = -1;
    S->cv_work.wait(lk, [&] {
      if (S->pending.empty()) return S->stopping;
      cls = next_class(S, &slot);
      return cls >= 0;
    });
    if (S->pending.empty() && S->stopping) break;
    // admit requests of that class, in arrival order, while device memory lasts
    std::vector<RequestP> batch;
    std::deque<RequestP> rest;
    size_t elems = 0;
    bool full = false;
    for (RequestP& r : S->pending) {
      const bool take = !full && (is_short(S, *r) ? 1 : 0) == cls;
      if (take && cls == 1 && elems + r->n > S->small_cut) full = true;
      if (take && cls == 0 && !batch.empty() && elems + r->n > S->long_cut) full = true;
      size_t off = 0;
      if (take && !full && batch.size() < kMaxBatchRequests &&
          (r->direct || S->arena->alloc(r->bytes, &off))) {
        r->off = off;
        elems += r->n;
        batch.push_back(r);
      } else {
        if (take) full = true;  // keep arrival order within the class
        rest.push_back(r);
      }
    }
    S->pending.swap(rest);
    if (batch.empty()) {  // memory is held by batches in flight: wait for one to finish
      S->cv_work.wait(lk);
      continue;
    }
    Slot& sl = S->slots[slot];
    sl.busy = true;
    sl.reqs = batch;
    lk.unlock();
    const cudaStream_t stream = cls == 1 ? sl.fast : sl.stream;
    // copy-in, one batched launch, copy-out
    IP_NVTX(cls == 1 ? "server batch (short requests)" : "server batch");
    int st = ISPRIME_OK;
    std::vector<isprime_array> arrays(batch.size());
    for (size_t i = 0; i < batch.size() && !st; ++i) {
      const Request& r = *batch[i];
      if (r.direct) {
        arrays[i] = {r.d_in, r.d_out, r.n};
        continue;
      }
      uint64_t* d_in = reinterpret_cast<uint64_t*>(S->d_arena + r.off);
      uint8_t* d_out = reinterpret_cast<uint8_t*>(S->d_arena + r.off + ((8 * r.n + 255) & ~(size_t)255));
      arrays[i] = {d_in, d_out, r.n};
      cudaError_t e = cudaMemcpyAsync(d_in, r.h_in, 8 * r.n, cudaMemcpyHostToDevice, stream);
      if (e != cudaSuccess) st = cuda_fail(e, "server copy-in");
    }
    if (!st) {
      std::lock_guard<std::mutex> cl(S->ctx->mu);  // host-side bookkeeping of the context
      // short batches (at most small_cut elements) run in the warp form
      st = batched_run(S->ctx, &sl.bs, arrays.data(), arrays.size(), cls == 1 ? S->small_cut : 0,
                       stream);
    }
    for (size_t i = 0; i < batch.size() && !st; ++i) {
      if (batch[i]->direct) continue;
      cudaError_t e = cudaMemcpyAsync(batch[i]->h_out, arrays[i].d_out, batch[i]->n,
                                      cudaMemcpyDeviceToHost, stream);
      if (e != cudaSuccess) st = cuda_fail(e, "server copy-out");
    }
    if (!st) {
      cudaError_t e = cudaEventRecord(sl.done_ev, stream);
      if (e != cudaSuccess) st = cuda_fail(e, "server event");
    }
    lk.lock();
    if (st) {  // the batch never reached the device: fail its requests now
      for (auto& r : batch)
        if (!r->direct) S->arena->release(r->off, r->bytes);
      fail_batch(sl, st);
      sl.reqs.clear();
      sl.busy = false;
      S->cv_done.notify_all();
      continue;
    }
    S->batches++;
    S->inflight.push_back(slot);
    S->cv_comp.notify_one();
  }
}

void completer_loop(isprime_server* S) {
  cudaSetDevice(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_comp.wait(lk, [&] { return !S->inflight.empty() || (S->stopping && S->pending.empty()); });
    if (S->inflight.empty()) {
      // stopping: leave once the dispatcher has nothing left either
      bool idle = true;
      for (auto& sl : S->slots) idle = idle && !sl.busy;
      if (idle) break;
      S->cv_comp.wait_for(lk, std::chrono::milliseconds(1));
      continue;
    }
    // poll every batch in flight; retire the finished ones
    std::vector<int> ready;
    for (int idx : S->inflight) {
      cudaError_t e = cudaEventQuery(S->slots[idx].done_ev);
      if (e == cudaSuccess) ready.push_back(idx);
      else if (e != cudaErrorNotReady) {
        S->fatal = cuda_fail(e, "server batch");
        ready.push_back(idx);
      }
    }
    if (ready.empty()) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
      continue;
    }
    const auto now = Clock::now();
    for (int idx : ready) {
      Slot& sl = S->slots[idx];
      for (auto& r : sl.reqs) {
        if (!r->direct) S->arena->release(r->off, r->bytes);
        r->status = S->fatal;
        r->done = true;
        S->latency_ms.push_back(std::chrono::duration<double, std::milli>(now - r->arrival).count());
        S->latency_short.push_back(is_short(S, *r) ? 1 : 0);
        S->elements += r->n;
        S->requests++;
      }
      S->last_done = now;
      sl.reqs.clear();
      sl.busy = false;
      S->inflight.erase(std::find(S->inflight.begin(), S->inflight.end(), idx));
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace
}  // namespace ip

using namespace ip;

extern "C" {

int isprime_server_create(isprime_ctx* ctx, size_t mem_budget_bytes, int n_slots,
                          isprime_server** out) {
  if (!ctx || !out) return set_error(ISPRIME_EINVAL, "NULL argument");
  if (mem_budget_bytes < (1u << 20)) return set_error(ISPRIME_EINVAL, "memory budget below 1 MiB");
  if (n_slots < 1 || n_slots > 16) return set_error(ISPRIME_EINVAL, "n_slots must be in [1, 16]");
  *out = nullptr;
  std::unique_ptr<isprime_server> S(new isprime_server());
  S->ctx = ctx;
  S->budget = mem_budget_bytes & ~(size_t)255;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    S->small_cut = ctx->tune.serve_short_max;
    S->long_cut = (size_t)1 << ctx->tune.serve_long_log2;
  }
  int prev = 0;
  IP_CUDA(cudaGetDevice(&prev));
  IP_CUDA(cudaSetDevice(ctx->device));
  int prio_lo = 0, prio_hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_arena, S->budget);
  if (e == cudaSuccess) {
    S->slots.resize(n_slots);
    for (auto& sl : S->slots) {
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&sl.fast, cudaStreamNonBlocking, prio_hi);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming);
    }
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    int st = cuda_fail(e, "server create");
    for (auto& sl : S->slots) {
      if (sl.stream) cudaStreamDestroy(sl.stream);
      if (sl.fast) cudaStreamDestroy(sl.fast);
      if (sl.done_ev) cudaEventDestroy(sl.done_ev);
    }
    cudaFree(S->d_arena);
    return st;
  }
  S->arena.reset(new Arena(S->budget));
  isprime_server* raw = S.get();
  S->dispatcher = std::thread(dispatcher_loop, raw);
  S->completer = std::thread(completer_loop, raw);
  *out = S.release();
  return ISPRIME_OK;
}

int isprime_server_submit(isprime_server* S, const uint64_t* h_in, uint8_t* h_out, size_t n,
                          uint64_t* ticket) {
  if (!S || !ticket) return set_error(ISPRIME_EINVAL, "NULL argument");
  if (n && (!h_in || !h_out)) return set_error(ISPRIME_EINVAL, "NULL pointer with n > 0");
  if (n && ((uintptr_t)h_in % 8)) return set_error(ISPRIME_EINVAL, "input not aligned to its element size");
  const size_t bytes = request_bytes(n);
  if (bytes > S->budget)
    return set_error(ISPRIME_EBUSY, "request needs " + std::to_string(bytes) +
                                        " bytes of device memory, more than the server budget");
  auto r = std::make_shared<Request>();
  r->h_in = h_in;
  r->h_out = h_out;
  r->n = n;
  r->bytes = bytes;
  r->arrival = Clock::now();
  void *din = nullptr, *dout = nullptr;
  if (n && n <= S->small_cut && device_view(h_in, &din) && device_view(h_out, &dout)) {
    r->direct = true;
    r->d_in = static_cast<const uint64_t*>(din);
    r->d_out = static_cast<uint8_t*>(dout);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stopping) return set_error(ISPRIME_EINVAL, "server is shutting down");
  r->ticket = S->next_ticket++;
  if (!S->any) {
    S->first_arrival = r->arrival;
    S->any = true;
  }
  S->tickets[r->ticket] = r;
  *ticket = r->ticket;
  if (n == 0) {
    r->done = true;
    S->latency_ms.push_back(0.0);
    S->latency_short.push_back(1);
    S->requests++;
    S->cv_done.notify_all();
    return ISPRIME_OK;
  }
  S->pending.push_back(r);
  S->cv_work.notify_one();
  return ISPRIME_OK;
}

int isprime_server_wait(isprime_server* S, uint64_t ticket, int timeout_ms) {
  if (!S) return set_error(ISPRIME_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return set_error(ISPRIME_EINVAL, "unknown or already collected ticket");
  RequestP r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms < 0) S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return set_error(ISPRIME_ETIMEDOUT, "request not finished within the timeout");
  S->tickets.erase(ticket);
  if (r->status) return set_error(r->status, "request failed on the device");
  return ISPRIME_OK;
}

int isprime_server_get_stats(isprime_server* S, isprime_server_stats* out) {
  if (!S || !out) return set_error(ISPRIME_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  isprime_server_stats st{};
  st.requests = S->requests;
  st.elements = S->elements;
  st.batches = S->batches;
  auto q = [](const std::vector<double>& v, double p) {
    return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))];
  };
  if (!S->latency_ms.empty()) {
    std::vector<double> v = S->latency_ms, vs, vl;
    for (size_t i = 0; i < v.size(); ++i) (S->latency_short[i] ? vs : vl).push_back(v[i]);
    std::sort(v.begin(), v.end());
    std::sort(vs.begin(), vs.end());
    std::sort(vl.begin(), vl.end());
    st.p50_ms = q(v, 0.50);
    st.p99_ms = q(v, 0.99);
    st.max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    st.mean_ms = sum / v.size();
    st.short_requests = vs.size();
    st.p50_short_ms = q(vs, 0.50);
    st.p99_short_ms = q(vs, 0.99);
    st.p50_long_ms = q(vl, 0.50);
    st.p99_long_ms = q(vl, 0.99);
  }
  if (S->any && S->requests) {
    st.span_s = std::chrono::duration<double>(S->last_done - S->first_arrival).count();
    st.tests_per_s = st.span_s > 0 ? S->elements / st.span_s : 0;
  }
  *out = st;
  return ISPRIME_OK;
}

int isprime_server_reset_stats(isprime_server* S) {
  if (!S) return set_error(ISPRIME_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  S->latency_ms.clear();
  S->latency_short.clear();
  S->requests = S->elements = S->batches = 0;
  S->any = false;
  return ISPRIME_OK;
}

int isprime_server_destroy(isprime_server* S) {
  if (!S) return ISPRIME_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  S->cv_comp.notify_all();
  S->dispatcher.join();
  S->cv_comp.notify_all();
  S->completer.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->ctx->device);
  for (auto& sl : S->slots) {
    cudaStreamSynchronize(sl.stream);
    cudaStreamSynchronize(sl.fast);
    batch_state_free(&sl.bs);
    cudaStreamDestroy(sl.stream);
    cudaStreamDestroy(sl.fast);
    cudaEventDestroy(sl.done_ev);
  }
  cudaFree(S->d_arena);
  cudaSetDevice(prev);
  delete S;
  return ISPRIME_OK;
}

}  // extern "C"
