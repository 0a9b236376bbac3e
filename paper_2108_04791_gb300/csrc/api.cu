// api.cu -- contexts and the C ABI declared in include/isprime.h.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>

#include "internal.h"

namespace ip {

static thread_local std::string t_last_error;

int set_error(int status, const std::string& msg) {
  t_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return set_error(e == cudaErrorMemoryAllocation ? ISPRIME_ENOMEM : ISPRIME_ECUDA, buf);
}

static cudaEvent_t pool_get(isprime_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int launch_begin(isprime_ctx* ctx, int kid, cudaStream_t s, TimedLaunch* tl) {
  tl->kid = kid;
  tl->start = tl->stop = nullptr;
  if (ctx->timing) {
    tl->start = pool_get(ctx);
    tl->stop = pool_get(ctx);
    if (!tl->start || !tl->stop) return set_error(ISPRIME_ECUDA, "cudaEventCreate failed");
    IP_CUDA(cudaEventRecord(tl->start, s));
  }
  return ISPRIME_OK;
}

int launch_end(isprime_ctx* ctx, cudaStream_t s, TimedLaunch* tl, const char* name) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, name);
  ctx->stats.kernel_launches++;
  if (ctx->timing) {
    IP_CUDA(cudaEventRecord(tl->stop, s));
    ctx->pending.push_back(*tl);
  }
  return ISPRIME_OK;
}

static int collect_timing(isprime_ctx* ctx) {
  for (auto& t : ctx->pending) {
    IP_CUDA(cudaEventSynchronize(t.stop));
    float ms = 0.f;
    IP_CUDA(cudaEventElapsedTime(&ms, t.start, t.stop));
    ctx->kernel_ms[t.kid] += ms;
    ctx->kernel_launches[t.kid] += 1;
    ctx->event_pool.push_back(t.start);
    ctx->event_pool.push_back(t.stop);
  }
  ctx->pending.clear();
  return ISPRIME_OK;
}

static isprime_tuning default_tuning() {
  isprime_tuning t{};
  t.classify_block = 256;
  t.mr_block = 256;
  t.blocks_per_sm = 32;  // classify 0.088 -> 0.086 ms on plain_large against 16
  t.td_primes = 15;  // 3..53
  t.chunk_log2 = 24;
  t.mont_impl = 9;       // formulation 6 with its correction on the multiply pipe:
  t.mont_impl_base2 = 9; // 0.8% / 1.0% faster than 6 on plain_large (six-base / base-2)
  t.batch_block = 128;
  t.batch_tile_log2 = 10;
  t.batch_blocks_per_sm = 0;
  t.base2_window = 1;
  t.rest_test = 0;
  t.small_max = 8192;
  t.compact_min = 33;
  t.sieve_cutover_log2 = 32;
  t.serve_short_max = 32768;
  // measured on plain_large (GB300): folds 2 and the s-split shorten the
  // step by 1.5% and 0.4%, 3-bit windows the six-base kernel by 1%, four
  // resident base-2 blocks per SM the base-2 kernel by 1.4%
  t.td_fold = 3;  // two residues: classify 0.106 -> 0.088 ms on plain_large
  t.base2_split = 1;
  t.base2_ilp = 1;
  t.rest_window = 3;
  t.window_ratio16 = 0;
  t.base2_blocks_per_sm = 4;
  t.pdl = 1;  // programmatic dependent launch of the Miller-Rabin kernels: 0.6% on plain_large
  t.td2_groups = 16;  // second trial stage, primes 59 .. 311: base 2 -12%, step -4.8% on plain_large
  t.dual_stream = 0;
  t.inplace_max_log2 = 0;
  t.serve_long_log2 = 24;
  t.rest_ilp = 2;  // six bases in pairs: six-base kernel -1.2% on plain_large
  t.host_chunk_log2 = 22;  // host path: 1.089 ms per 2^24 values against 1.26 (23) and 1.15 (21)
  return t;
}

static int check_tuning(const isprime_tuning& t) {
  auto bad_block = [](uint32_t b, uint32_t maxb) { return b < 32 || b > maxb || (b % 32) != 0; };
  if (bad_block(t.classify_block, 1024)) return set_error(ISPRIME_EINVAL, "classify_block must be a multiple of 32 in [32, 1024]");
  if (bad_block(t.mr_block, 256)) return set_error(ISPRIME_EINVAL, "mr_block must be a multiple of 32 in [32, 256]");
  if (t.blocks_per_sm < 1 || t.blocks_per_sm > 32) return set_error(ISPRIME_EINVAL, "blocks_per_sm must be in [1, 32]");
  if (t.td_primes > 53) return set_error(ISPRIME_EINVAL, "td_primes must be in [0, 53]");
  if (t.chunk_log2 < 16 || t.chunk_log2 > 28) return set_error(ISPRIME_EINVAL, "chunk_log2 must be in [16, 28]");
  if (t.mont_impl > 9) return set_error(ISPRIME_EINVAL, "mont_impl must be in [0, 9]");
  if (t.mont_impl_base2 > 9) return set_error(ISPRIME_EINVAL, "mont_impl_base2 must be in [0, 9]");
  if (bad_block(t.batch_block, 256)) return set_error(ISPRIME_EINVAL, "batch_block must be a multiple of 32 in [32, 256]");
  if (t.batch_tile_log2 < 8 || t.batch_tile_log2 > 14) return set_error(ISPRIME_EINVAL, "batch_tile_log2 must be in [8, 14]");
  if (t.batch_blocks_per_sm > 32) return set_error(ISPRIME_EINVAL, "batch_blocks_per_sm must be in [0, 32]");
  if (t.base2_window != 0 && t.base2_window != 1 && t.base2_window != 2 && t.base2_window != 4)
    return set_error(ISPRIME_EINVAL, "base2_window must be 0, 1, 2 or 4");
  if (t.rest_test > 1) return set_error(ISPRIME_EINVAL, "rest_test must be 0 or 1");
  if (t.small_max > (1u << 20)) return set_error(ISPRIME_EINVAL, "small_max must be in [0, 2^20]");
  if (t.compact_min > 33) return set_error(ISPRIME_EINVAL, "compact_min must be in [0, 33]");
  if (t.sieve_cutover_log2 > 32) return set_error(ISPRIME_EINVAL, "sieve_cutover_log2 must be in [0, 32]");
  if (t.serve_short_max > (1u << 20)) return set_error(ISPRIME_EINVAL, "serve_short_max must be in [0, 2^20]");
  if (t.td_fold > 3) return set_error(ISPRIME_EINVAL, "td_fold must be in [0, 3]");
  if (t.base2_split > 1) return set_error(ISPRIME_EINVAL, "base2_split must be 0 or 1");
  if (t.base2_ilp != 1 && t.base2_ilp != 2) return set_error(ISPRIME_EINVAL, "base2_ilp must be 1 or 2");
  if (t.rest_window != 3 && t.rest_window != 4) return set_error(ISPRIME_EINVAL, "rest_window must be 3 or 4");
  if (t.window_ratio16 > 4096) return set_error(ISPRIME_EINVAL, "window_ratio16 must be in [0, 4096]");
  if (t.base2_blocks_per_sm > 32) return set_error(ISPRIME_EINVAL, "base2_blocks_per_sm must be in [0, 32]");
  if (t.pdl > 1) return set_error(ISPRIME_EINVAL, "pdl must be 0 or 1");
  if (t.dual_stream > 1) return set_error(ISPRIME_EINVAL, "dual_stream must be 0 or 1");
  if (t.inplace_max_log2 > 24) return set_error(ISPRIME_EINVAL, "inplace_max_log2 must be <= 24");
  if (t.rest_ilp < 1 || t.rest_ilp > 2) return set_error(ISPRIME_EINVAL, "rest_ilp must be 1 or 2");
  if (t.serve_long_log2 < 16 || t.serve_long_log2 > 28)
    return set_error(ISPRIME_EINVAL, "serve_long_log2 must be in [16, 28]");
  if (t.host_chunk_log2 < 16 || t.host_chunk_log2 > 24)
    return set_error(ISPRIME_EINVAL, "host_chunk_log2 must be in [16, 24]");
  if (t.td2_groups != 0 && t.td2_groups != 8 && t.td2_groups != 12 && t.td2_groups != 16 &&
      t.td2_groups != 24)
    return set_error(ISPRIME_EINVAL, "td2_groups must be 0, 8, 12, 16 or 24");
  return ISPRIME_OK;
}

static void free_queues(Queues& q) {
  cudaFree(q.q64_n);
  cudaFree(q.q64_idx);
  cudaFree(q.q64b);
  cudaFree(q.q32_n);
  cudaFree(q.q32_idx);
  cudaFree(q.counters);
  q = Queues{};
}

static int alloc_queues(Queues* out, size_t cap) {
  Queues q;
  IP_CUDA(cudaMalloc(&q.q64_n, cap * sizeof(uint64_t)));
  IP_CUDA(cudaMalloc(&q.q64_idx, cap * sizeof(uint32_t)));
  IP_CUDA(cudaMalloc(&q.q64b, cap * sizeof(uint32_t)));
  IP_CUDA(cudaMalloc(&q.q32_n, cap * sizeof(uint32_t)));
  IP_CUDA(cudaMalloc(&q.q32_idx, cap * sizeof(uint32_t)));
  IP_CUDA(cudaMalloc(&q.counters, kQueueCounters * sizeof(uint32_t)));
  q.capacity = cap;
  *out = q;
  return ISPRIME_OK;
}

static int ensure_queues(isprime_ctx* ctx, size_t cap) {
  if (ctx->q.capacity >= cap) return ISPRIME_OK;
  if (ctx->order_ev_valid) IP_CUDA(cudaEventSynchronize(ctx->order_ev));
  free_queues(ctx->q);
  return alloc_queues(&ctx->q, cap);
}

// The second queue set, stream and fork/join events of the two-stream form.
static int ensure_dual(isprime_ctx* ctx, size_t cap) {
  if (!ctx->dual_s) {
    IP_CUDA(cudaStreamCreateWithFlags(&ctx->dual_s, cudaStreamNonBlocking));
    IP_CUDA(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
    IP_CUDA(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming));
  }
  if (ctx->q2.capacity >= cap) return ISPRIME_OK;
  if (ctx->order_ev_valid) IP_CUDA(cudaEventSynchronize(ctx->order_ev));
  free_queues(ctx->q2);
  return alloc_queues(&ctx->q2, cap);
}

static size_t scratch_bytes(const isprime_ctx* ctx) {
  return ctx->sieve_limit / 16 +
         (ctx->q.capacity + ctx->q2.capacity + ctx->host_q[0].capacity +
          ctx->host_q[1].capacity) * 24 +
         ctx->stage_elems * 9 * isprime_ctx::kStageSlots + 2 * sizeof(unsigned long long) +
         ctx->window_cap;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

static int ctx_create(int device, uint64_t sieve_limit, isprime_ctx** out) {
  if (!out) return set_error(ISPRIME_EINVAL, "out is NULL");
  *out = nullptr;
  if (sieve_limit == ISPRIME_SIEVE_DEFAULT) sieve_limit = 1ull << 32;
  if (sieve_limit > (1ull << 32) || (sieve_limit & ((1ull << 20) - 1)) != 0)
    return set_error(ISPRIME_EINVAL, "sieve_limit must be 0 or a multiple of 2^20 no larger than 2^32");
  int ndev = 0;
  IP_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(ISPRIME_EINVAL, "device out of range");
  DeviceGuard g(device);
  std::unique_ptr<isprime_ctx> ctx(new isprime_ctx());
  ctx->device = device;
  IP_CUDA(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
  IP_CUDA(cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  ctx->tune = default_tuning();
  ctx->sieve_limit = sieve_limit;
  IP_CUDA(cudaEventCreateWithFlags(&ctx->order_ev, cudaEventDisableTiming));
  IP_CUDA(cudaEventCreateWithFlags(&ctx->f64_ev, cudaEventDisableTiming));
  IP_CUDA(cudaMalloc(&ctx->d_status, 2 * sizeof(unsigned long long)));
  IP_CUDA(cudaMemset(ctx->d_status, 0, 2 * sizeof(unsigned long long)));
  cudaStream_t s;
  IP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  int st = ISPRIME_OK;
  if (sieve_limit) {
    cudaError_t e = cudaMalloc(&ctx->d_sieve, sieve_limit / 16);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc(sieve)");
  }
  if (!st) st = sieve_build(ctx.get(), s);
  if (!st) st = ensure_queues(ctx.get(), (size_t)1 << 20);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (st) {
    isprime_ctx_destroy(ctx.release());
    return st;
  }
  *out = ctx.release();
  return ISPRIME_OK;
}

// Orders this call's use of the shared scratch after the previous call's,
// whatever stream that was on.
static int order_before(isprime_ctx* ctx, cudaStream_t s) {
  if (ctx->order_ev_valid) IP_CUDA(cudaStreamWaitEvent(s, ctx->order_ev, 0));
  return ISPRIME_OK;
}
static int order_after(isprime_ctx* ctx, cudaStream_t s) {
  IP_CUDA(cudaEventRecord(ctx->order_ev, s));
  ctx->order_ev_valid = true;
  return ISPRIME_OK;
}

// The double-path calls of a context form one chain (each waits for the
// previous one's kernels), so that isprime_f64_sync_status, which waits for
// the chain's last event, sees the counts of every earlier call.
static int f64_before(isprime_ctx* ctx, cudaStream_t s) {
  if (ctx->f64_ev_valid) IP_CUDA(cudaStreamWaitEvent(s, ctx->f64_ev, 0));
  return ISPRIME_OK;
}
static int f64_after(isprime_ctx* ctx, cudaStream_t s) {
  IP_CUDA(cudaEventRecord(ctx->f64_ev, s));
  ctx->f64_ev_valid = true;
  return ISPRIME_OK;
}

static bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t a0 = (uintptr_t)a, a1 = a0 + na, b0 = (uintptr_t)b, b1 = b0 + nb;
  return a0 < b1 && b0 < a1;
}

// The array path: classify + Miller-Rabin per chunk, all asynchronous.
// Argument checks shared by every array entry point (no CUDA calls).
static int check_array_args(const void* d_in, const void* d_out, size_t n, size_t esz) {
  if (n == 0) return ISPRIME_OK;
  if (!d_in || !d_out) return set_error(ISPRIME_EINVAL, "NULL pointer with n > 0");
  if ((uintptr_t)d_in % esz) return set_error(ISPRIME_EINVAL, "input not aligned to its element size");
  if (n > (SIZE_MAX / esz)) return set_error(ISPRIME_EINVAL, "n too large");
  if (ranges_overlap(d_in, n * esz, d_out, n)) return set_error(ISPRIME_EINVAL, "output overlaps input");
  return ISPRIME_OK;
}

// One chunk (len <= q.capacity) through the queue path: classify, then the
// Miller-Rabin stages on the queues q, all on stream s.  The caller holds
// ctx->mu and orders the uses of q.
template <bool kF64>
static int run_chunk(isprime_ctx* ctx, const Queues& q, const void* in, uint8_t* out, size_t len,
                     unsigned long long* d_invalid, cudaStream_t s) {
  IP_CUDA(cudaMemsetAsync(q.counters, 0, kQueueCounters * sizeof(uint32_t), s));
  ClassifyArgs a;
  a.in = in;
  a.out = out;
  a.n = len;
  a.sieve = ctx->d_sieve;
  a.sieve_limit = sieve_cut(ctx);
  a.ntd = ctx->tune.td_primes;
  a.td_square = td_square_for(ctx->tune.td_primes);
  a.q64_n = q.q64_n;
  a.q64_idx = q.q64_idx;
  a.q32_n = q.q32_n;
  a.q32_idx = q.q32_idx;
  a.counters = q.counters;
  a.invalid = d_invalid;
  a.invalid_ctx = kF64 ? ctx->d_status : nullptr;
  a.head = ((uintptr_t)a.in % 16) ? 1u : 0u;
  if (a.head > len) a.head = (uint32_t)len;
  a.pair_store = (((uintptr_t)(a.out + a.head)) % 2 == 0) ? 1u : 0u;
  a.q64_cap = (uint32_t)q.capacity;
  a.fold = ctx->tune.td_fold;
  a.split = ctx->tune.base2_split;
  int st = kF64 ? launch_classify_f64(ctx, a, s) : launch_classify_u64(ctx, a, s);
  if (st) return st;
  return launch_mr(ctx, q, a.out, len, s);
}

template <bool kF64>
static int run_array(isprime_ctx* ctx, const void* d_in, uint8_t* d_out, size_t n,
                     unsigned long long* d_invalid, cudaStream_t s) {
  const size_t esz = 8;
  if (n == 0) return ISPRIME_OK;
  int st0 = check_array_args(d_in, d_out, n, esz);
  if (st0) return st0;
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  int st;
  if (n <= ctx->tune.small_max) {  // one launch, no queues: no ordering needed
    if (kF64 && (st = f64_before(ctx, s))) return st;
    st = kF64 ? launch_small_f64(ctx, static_cast<const double*>(d_in), d_out, n, d_invalid,
                                 ctx->d_status, s)
              : launch_small_u64(ctx, static_cast<const uint64_t*>(d_in), d_out, n, s);
    if (st) return st;
    if (kF64 && (st = f64_after(ctx, s))) return st;
    ctx->stats.calls++;
    ctx->stats.elements += n;
    return ISPRIME_OK;
  }
  size_t chunk = (size_t)1 << ctx->tune.chunk_log2;
  // Two-stream form: at least two chunks, alternating between the caller's
  // stream with the context's queues and a second stream with a second queue
  // set, so that one chunk's classify overlaps the other's Miller-Rabin
  // kernels and each kernel's last wave is filled by the other stream's.
  const bool dual = ctx->tune.dual_stream != 0 && n >= ((size_t)1 << 20);
  if (dual) chunk = std::min(chunk, ((n + 1) / 2 + 0xFFFF) & ~(size_t)0xFFFF);
  st = ensure_queues(ctx, std::min(chunk, std::max(n, (size_t)1 << 16)));
  if (st) return st;
  if (dual && (st = ensure_dual(ctx, std::min(chunk, ctx->q.capacity)))) return st;
  if ((st = order_before(ctx, s))) return st;
  if (kF64 && (st = f64_before(ctx, s))) return st;
  if (!kF64) {  // the window path, when the tuning asks for the per-call choice
    bool taken = false;
    if ((st = window_try(ctx, static_cast<const uint64_t*>(d_in), d_out, n, s, &taken))) return st;
    if (taken) {
      if ((st = order_after(ctx, s))) return st;
      ctx->stats.calls++;
      ctx->stats.elements += n;
      return ISPRIME_OK;
    }
  }
  const size_t step = std::min(chunk, dual ? std::min(ctx->q.capacity, ctx->q2.capacity)
                                            : ctx->q.capacity);
  if (dual) {  // the second stream starts after everything the caller's stream holds
    IP_CUDA(cudaEventRecord(ctx->fork_ev, s));
    IP_CUDA(cudaStreamWaitEvent(ctx->dual_s, ctx->fork_ev, 0));
  }
  size_t k = 0;
  st = ISPRIME_OK;
  for (size_t off = 0; off < n && !st; off += step, ++k) {
    const size_t len = std::min(step, n - off);
    const bool second = dual && (k & 1);
    st = run_chunk<kF64>(ctx, second ? ctx->q2 : ctx->q, static_cast<const char*>(d_in) + off * esz,
                         d_out + off, len, d_invalid, second ? ctx->dual_s : s);
  }
  if (dual) {  // and the caller's stream continues after both (also after a failed launch)
    IP_CUDA(cudaEventRecord(ctx->join_ev, ctx->dual_s));
    IP_CUDA(cudaStreamWaitEvent(s, ctx->join_ev, 0));
  }
  if (st) return st;
  if (kF64 && (st = f64_after(ctx, s))) return st;
  if ((st = order_after(ctx, s))) return st;
  ctx->stats.calls++;
  ctx->stats.elements += n;
  return ISPRIME_OK;
}

// Take-and-clear of the context's invalid-element count (one thread).
__global__ void take_invalid_kernel(unsigned long long* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) status[1] = atomicExch(&status[0], 0ull);
}

// ---------------------------------------------------------------- defaults

static std::mutex g_default_mu;
static isprime_ctx* g_default[64] = {};

static int default_ctx(int device, isprime_ctx** out) {
  if (device < 0 || device >= 64) return set_error(ISPRIME_EINVAL, "device out of range");
  std::lock_guard<std::mutex> lock(g_default_mu);
  if (!g_default[device]) {
    int st = ctx_create(device, ISPRIME_SIEVE_DEFAULT, &g_default[device]);
    if (st) return st;
  }
  *out = g_default[device];
  return ISPRIME_OK;
}

static int current_default(isprime_ctx** out) {
  int dev = 0;
  IP_CUDA(cudaGetDevice(&dev));
  return default_ctx(dev, out);
}

}  // namespace ip

using namespace ip;

extern "C" {

int isprime_ctx_create(int device, uint64_t sieve_limit, isprime_ctx** out) {
  return ctx_create(device, sieve_limit, out);
}

int isprime_ctx_destroy(isprime_ctx* ctx) {
  if (!ctx) return ISPRIME_OK;
  {
    DeviceGuard g(ctx->device);
    if (ctx->order_ev_valid) cudaEventSynchronize(ctx->order_ev);
    collect_timing(ctx);
    free_queues(ctx->q);
    free_queues(ctx->q2);
    if (ctx->dual_s) cudaStreamSynchronize(ctx->dual_s), cudaStreamDestroy(ctx->dual_s);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    cudaFree(ctx->d_sieve);
    cudaFree(ctx->d_base_primes);
    cudaFree(ctx->d_nprimes);
    cudaFree(ctx->d_stage_in);
    cudaFree(ctx->d_stage_out);
    if (ctx->h_pin_in) cudaFreeHost(ctx->h_pin_in);
    if (ctx->h_pin_out) cudaFreeHost(ctx->h_pin_out);
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    batch_state_free(&ctx->batch);
    for (auto e : ctx->stage_ev)
      if (e) cudaEventDestroy(e);
    if (ctx->host_last) cudaEventDestroy(ctx->host_last);
    if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
    if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
    for (auto& hs : ctx->host_s)
      if (hs) cudaStreamDestroy(hs);
    for (auto& hq : ctx->host_q) free_queues(hq);
    if (ctx->order_ev) cudaEventDestroy(ctx->order_ev);
    if (ctx->f64_ev) cudaEventDestroy(ctx->f64_ev);
    if (ctx->status_s) cudaStreamSynchronize(ctx->status_s), cudaStreamDestroy(ctx->status_s);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_mm);
    if (ctx->h_mm) cudaFreeHost(ctx->h_mm);
    cudaFree(ctx->d_window);
    if (ctx->scalar_s) cudaStreamSynchronize(ctx->scalar_s), cudaStreamDestroy(ctx->scalar_s);
    if (ctx->h_inline_out) cudaFreeHost(ctx->h_inline_out);
  }
  for (int d = 0; d < 64; ++d) {
    std::lock_guard<std::mutex> lock(g_default_mu);
    if (g_default[d] == ctx) g_default[d] = nullptr;
  }
  delete ctx;
  return ISPRIME_OK;
}

int isprime_default_ctx(int device, isprime_ctx** out) {
  if (!out) return set_error(ISPRIME_EINVAL, "out is NULL");
  return default_ctx(device, out);
}

int isprime_tuning_defaults(isprime_tuning* out) {
  if (!out) return set_error(ISPRIME_EINVAL, "NULL argument");
  *out = default_tuning();
  return ISPRIME_OK;
}

int isprime_ctx_get_tuning(const isprime_ctx* ctx, isprime_tuning* out) {
  if (!ctx || !out) return set_error(ISPRIME_EINVAL, "NULL argument");
  *out = ctx->tune;
  return ISPRIME_OK;
}

int isprime_ctx_set_tuning(isprime_ctx* ctx, const isprime_tuning* t) {
  if (!ctx || !t) return set_error(ISPRIME_EINVAL, "NULL argument");
  int st = check_tuning(*t);
  if (st) return st;
  const size_t smem = batched_smem_bytes(t->batch_block, 1u << t->batch_tile_log2);
  if (smem > (size_t)ctx->smem_optin)
    return set_error(ISPRIME_EINVAL, "batch_block and batch_tile_log2 need " + std::to_string(smem) +
                                         " bytes of shared memory per block; this GPU allows " +
                                         std::to_string(ctx->smem_optin));
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->tune = *t;
  return ISPRIME_OK;
}

int isprime_ctx_stats(const isprime_ctx* ctx, isprime_stats* out) {
  if (!ctx || !out) return set_error(ISPRIME_EINVAL, "NULL argument");
  *out = ctx->stats;
  out->sieve_limit = ctx->sieve_limit;
  out->scratch_bytes = scratch_bytes(ctx);
  return ISPRIME_OK;
}

int isprime_u64_ctx(isprime_ctx* ctx, const uint64_t* d_in, uint8_t* d_out, size_t n,
                    isprime_stream stream) {
  IP_NVTX("isprime_u64_ctx");
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  return run_array<false>(ctx, d_in, d_out, n, nullptr, (cudaStream_t)stream);
}

int isprime_u64(const uint64_t* d_in, uint8_t* d_out, size_t n, isprime_stream stream) {
  IP_NVTX("isprime_u64");
  if (n == 0) return ISPRIME_OK;
  int st = check_array_args(d_in, d_out, n, 8);
  if (st) return st;
  isprime_ctx* ctx = nullptr;
  st = current_default(&ctx);
  if (st) return st;
  return run_array<false>(ctx, d_in, d_out, n, nullptr, (cudaStream_t)stream);
}

int isprime_f64_ctx(isprime_ctx* ctx, const double* d_in, uint8_t* d_out, size_t n,
                    unsigned long long* d_invalid, isprime_stream stream) {
  IP_NVTX("isprime_f64_ctx");
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  return run_array<true>(ctx, d_in, d_out, n, d_invalid, (cudaStream_t)stream);
}

int isprime_f64(const double* d_in, uint8_t* d_out, size_t n, unsigned long long* d_invalid,
                isprime_stream stream) {
  IP_NVTX("isprime_f64");
  if (n == 0) return ISPRIME_OK;
  int st = check_array_args(d_in, d_out, n, 8);
  if (st) return st;
  isprime_ctx* ctx = nullptr;
  st = current_default(&ctx);
  if (st) return st;
  return run_array<true>(ctx, d_in, d_out, n, d_invalid, (cudaStream_t)stream);
}

int isprime_f64_sync_status(isprime_ctx* ctx, unsigned long long* count) {
  IP_NVTX("isprime_f64_sync_status");
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  if (count) *count = 0;
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  if (!ctx->status_s) IP_CUDA(cudaStreamCreateWithFlags(&ctx->status_s, cudaStreamNonBlocking));
  if (ctx->f64_ev_valid) IP_CUDA(cudaStreamWaitEvent(ctx->status_s, ctx->f64_ev, 0));
  take_invalid_kernel<<<1, 32, 0, ctx->status_s>>>(ctx->d_status);
  IP_CUDA(cudaGetLastError());
  unsigned long long v = 0;
  IP_CUDA(cudaMemcpyAsync(&v, ctx->d_status + 1, sizeof v, cudaMemcpyDeviceToHost, ctx->status_s));
  IP_CUDA(cudaStreamSynchronize(ctx->status_s));
  if (count) *count = v;
  if (v == 0) return ISPRIME_OK;
  return set_error(ISPRIME_EDOMAIN, std::to_string(v) +
                                        " double input(s) were not integers in [0, 2^53] (output 0)");
}

int isprime_range(isprime_ctx* ctx, uint64_t lo, uint64_t count, uint8_t* d_out,
                  isprime_stream stream) {
  IP_NVTX("isprime_range");
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  if (count == 0) return ISPRIME_OK;
  if (!d_out) return set_error(ISPRIME_EINVAL, "d_out is NULL with count > 0");
  if (count - 1 > UINT64_MAX - lo) return set_error(ISPRIME_EINVAL, "lo + count exceeds 2^64");
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  const size_t chunk = (size_t)1 << ctx->tune.chunk_log2;
  int st = ensure_queues(ctx, std::min(chunk, std::max((size_t)std::min<uint64_t>(count, chunk),
                                                       (size_t)kRangeChunkAlign)));
  if (st) return st;
  if ((st = order_before(ctx, s))) return st;
  if ((st = range_run(ctx, lo, count, d_out, s))) return st;
  if ((st = order_after(ctx, s))) return st;
  ctx->stats.calls++;
  ctx->stats.elements += count;
  return ISPRIME_OK;
}

int isprime_u64_batched(isprime_ctx* ctx, const isprime_array* arrays, size_t n_arrays,
                        isprime_stream stream) {
  IP_NVTX("isprime_u64_batched");
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  if (n_arrays == 0) return ISPRIME_OK;
  if (!arrays) return set_error(ISPRIME_EINVAL, "arrays is NULL");
  for (size_t i = 0; i < n_arrays; ++i) {
    int st = check_array_args(arrays[i].d_in, arrays[i].d_out, arrays[i].n, 8);
    if (st) return set_error(st, "array " + std::to_string(i) + ": " + t_last_error);
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  int st = order_before(ctx, s);
  if (st) return st;
  if ((st = batched_run(ctx, &ctx->batch, arrays, n_arrays, ctx->tune.small_max, s))) return st;
  if ((st = order_after(ctx, s))) return st;
  ctx->stats.calls++;
  return ISPRIME_OK;
}

int isprime_u64_scalar(isprime_ctx* ctx, uint64_t value, uint8_t* result) {
  IP_NVTX("isprime_u64_scalar");
  if (!ctx || !result) return set_error(ISPRIME_EINVAL, "NULL argument");
  DeviceGuard g(ctx->device);
  {
    std::lock_guard<std::mutex> lock(ctx->inline_mu);
    if (!ctx->scalar_s) IP_CUDA(cudaStreamCreateWithFlags(&ctx->scalar_s, cudaStreamNonBlocking));
  }
  return inline_run(ctx, &value, result, 1, ctx->scalar_s);
}

int isprime_u64_host(isprime_ctx* ctx, const uint64_t* h_in, uint8_t* h_out, size_t n,
                     isprime_stream stream) {
  IP_NVTX("isprime_u64_host");
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  if (n == 0) return ISPRIME_OK;
  int st = check_array_args(h_in, h_out, n, 8);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(ctx->device);
  if (n <= (size_t)kInlineMax) return inline_run(ctx, h_in, h_out, n, s);
  std::lock_guard<std::mutex> host_lock(ctx->host_mu);
  // Pipeline: chunk k is copied in on copy_in into staging slot k % 4,
  // classified on compute stream k % 2 with that stream's own queues, and
  // copied out on copy_out.  With four staging slots the copy engine runs up
  // to two chunks ahead of the kernels (a slot is refilled once the chunk
  // four back has been computed and copied out), so after the first chunk
  // the kernels rarely wait for a copy; the kernels of consecutive chunks, on
  // the two streams, overlap each other's tails.
  constexpr int kSlots = isprime_ctx::kStageSlots;
  const size_t step_max =
      std::min((size_t)1 << ctx->tune.chunk_log2, (size_t)1 << ctx->tune.host_chunk_log2);
  const size_t stage = std::min(step_max, n);
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->copy_in) {
      IP_CUDA(cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking));
      IP_CUDA(cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking));
      for (auto& hs : ctx->host_s) IP_CUDA(cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking));
      for (auto& e : ctx->stage_ev) IP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      IP_CUDA(cudaEventCreateWithFlags(&ctx->host_last, cudaEventDisableTiming));
    }
    // Earlier host-path calls have finished (each one waits before returning).
    for (auto& hq : ctx->host_q)
      if (hq.capacity < stage) {
        free_queues(hq);
        if ((st = alloc_queues(&hq, stage))) return st;
      }
    if (ctx->stage_elems < stage) {
      if (ctx->order_ev_valid) IP_CUDA(cudaEventSynchronize(ctx->order_ev));
      cudaFree(ctx->d_stage_in);
      cudaFree(ctx->d_stage_out);
      ctx->d_stage_in = nullptr;
      ctx->d_stage_out = nullptr;
      ctx->stage_elems = 0;
      IP_CUDA(cudaMalloc(&ctx->d_stage_in, kSlots * stage * sizeof(uint64_t)));
      IP_CUDA(cudaMalloc(&ctx->d_stage_out, kSlots * stage));
      ctx->stage_elems = stage;
    }
  }
  const size_t step = std::min(ctx->stage_elems, step_max);
  cudaEvent_t* in_ready = &ctx->stage_ev[0];            // copy-in of a slot finished
  cudaEvent_t* comp_done = &ctx->stage_ev[kSlots];      // kernels on a slot finished
  cudaEvent_t* out_done = &ctx->stage_ev[2 * kSlots];   // copy-out of a slot finished
  // The slots may still be in use by a previous call's last chunks.
  IP_CUDA(cudaStreamWaitEvent(ctx->copy_in, ctx->host_last, 0));
  // Arrays of at least four full chunks start with a quarter and a half of a
  // full chunk, so that the kernels start after a short first copy and the
  // pipeline fills sooner (measured: 13.6 against 13.1 G tests/s on 2^24
  // values; an eighth first was slower again); shorter arrays would only pay
  // the extra launches.  The rest of the array is cut into equal chunks of at
  // most a full one, so no short chunk is left at the end.
  const bool ramp_up = n >= 4 * step;
  const size_t ramp = ramp_up ? step / 4 + step / 2 : 0;
  const size_t rest_chunks = (n - ramp + step - 1) / step;
  const size_t even = (n - ramp + rest_chunks - 1) / rest_chunks;
  for (size_t off = 0, k = 0, len = 0; off < n; off += len, ++k) {
    const size_t want = ramp_up && k == 0 ? step / 4 : ramp_up && k == 1 ? step / 2 : even;
    len = std::min(want, n - off);
    const int slot = (int)(k % kSlots);
    const int lane = (int)(k & 1);  // compute stream and queue set
    uint64_t* din = ctx->d_stage_in + slot * step;
    uint8_t* dout = ctx->d_stage_out + slot * step;
    if (k >= (size_t)kSlots) IP_CUDA(cudaStreamWaitEvent(ctx->copy_in, comp_done[slot], 0));
    IP_CUDA(cudaMemcpyAsync(din, h_in + off, len * 8, cudaMemcpyHostToDevice, ctx->copy_in));
    IP_CUDA(cudaEventRecord(in_ready[slot], ctx->copy_in));
    const cudaStream_t cs = ctx->host_s[lane];
    IP_CUDA(cudaStreamWaitEvent(cs, in_ready[slot], 0));
    if (k >= (size_t)kSlots) IP_CUDA(cudaStreamWaitEvent(cs, out_done[slot], 0));
    {
      std::lock_guard<std::mutex> lock(ctx->mu);
      st = len <= ctx->tune.small_max
               ? launch_small_u64(ctx, din, dout, len, cs)
               : run_chunk<false>(ctx, ctx->host_q[lane], din, dout, len, nullptr, cs);
    }
    if (st) return st;
    IP_CUDA(cudaEventRecord(comp_done[slot], cs));
    IP_CUDA(cudaStreamWaitEvent(ctx->copy_out, comp_done[slot], 0));
    IP_CUDA(cudaMemcpyAsync(h_out + off, dout, len, cudaMemcpyDeviceToHost, ctx->copy_out));
    IP_CUDA(cudaEventRecord(out_done[slot], ctx->copy_out));
  }
  IP_CUDA(cudaEventRecord(ctx->host_last, ctx->copy_out));
  // copy_out waited for every chunk's kernels, so this is the end of the call
  IP_CUDA(cudaStreamSynchronize(ctx->copy_out));
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->stats.calls++;
    ctx->stats.elements += n;
  }
  return ISPRIME_OK;
}

int isprime_sieve_count(isprime_ctx* ctx, uint64_t* out) {
  IP_NVTX("isprime_sieve_count");
  if (!ctx || !out) return set_error(ISPRIME_EINVAL, "NULL argument");
  *out = 0;
  if (ctx->sieve_limit == 0) return ISPRIME_OK;
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  uint64_t* d = nullptr;
  IP_CUDA(cudaMalloc(&d, sizeof(uint64_t)));
  cudaStream_t s;
  IP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  IP_CUDA(cudaMemsetAsync(d, 0, sizeof(uint64_t), s));
  int st = sieve_count(ctx, s, d);
  uint64_t h = 0;
  if (!st) {
    cudaError_t e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "sieve count readback");
  }
  cudaStreamDestroy(s);
  cudaFree(d);
  if (st) return st;
  *out = h + (ctx->sieve_limit > 2 ? 1 : 0);  // the bitmap holds odd numbers; add the prime 2
  return ISPRIME_OK;
}

int isprime_timing_enable(isprime_ctx* ctx, int on) {
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->timing = on != 0;
  return ISPRIME_OK;
}

int isprime_timing_read(isprime_ctx* ctx, isprime_kernel_time* out, int count) {
  if (!ctx || !out) return set_error(ISPRIME_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  int st = collect_timing(ctx);
  if (st) return st;
  for (int k = 0; k < count && k < ISPRIME_K_COUNT; ++k) {
    out[k].total_ms = ctx->kernel_ms[k];
    out[k].launches = ctx->kernel_launches[k];
  }
  return ISPRIME_OK;
}

int isprime_timing_reset(isprime_ctx* ctx) {
  if (!ctx) return set_error(ISPRIME_EINVAL, "ctx is NULL");
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard g(ctx->device);
  int st = collect_timing(ctx);
  for (int k = 0; k < ISPRIME_K_COUNT; ++k) {
    ctx->kernel_ms[k] = 0;
    ctx->kernel_launches[k] = 0;
  }
  return st;
}

int isprime_count_ops(isprime_ctx* ctx, const uint64_t* d_in, uint8_t* d_out, size_t n,
                      isprime_op_counts* out) {
  IP_NVTX("isprime_count_ops");
  if (!ctx || !out) return set_error(ISPRIME_EINVAL, "NULL argument");
  memset(out, 0, sizeof *out);
  int st = check_array_args(d_in, d_out, n, 8);
  if (st || n == 0) return st;
  DeviceGuard g(ctx->device);
  unsigned long long c[2][3][2];
  isprime_tuning saved;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->order_ev_valid) IP_CUDA(cudaEventSynchronize(ctx->order_ev));
    if ((st = op_counts_read(c, true))) return st;
    saved = ctx->tune;
    ctx->tune.small_max = 0;  // the queue path, whose kernels count
    ctx->count_ops = true;
  }
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    st = run_array<false>(ctx, d_in, d_out, n, nullptr, s);
    e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  {
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->count_ops = false;
    ctx->tune = saved;
  }
  if (e != cudaSuccess) return cuda_fail(e, "isprime_count_ops stream");
  if (st) return st;
  if ((st = op_counts_read(c, true))) return st;
  out->elements = n;
  out->base2_squarings[0] = c[0][0][0];
  out->base2_squarings[1] = c[0][0][1];
  out->base2_products[0] = c[0][1][0];
  out->base2_products[1] = c[0][1][1];
  out->base2_steps[0] = c[0][2][0];
  out->base2_steps[1] = c[0][2][1];
  out->rest_squarings[0] = c[1][0][0];
  out->rest_squarings[1] = c[1][0][1];
  out->rest_products[0] = c[1][1][0];
  out->rest_products[1] = c[1][1][1];
  return ISPRIME_OK;
}

int isprime_debug_checks(int reset, uint32_t* sites, uint64_t* violations, int* compiled) {
  if (!sites || !violations) return set_error(ISPRIME_EINVAL, "NULL argument");
#if defined(IP_DEBUG_CHECKS)
  if (compiled) *compiled = 1;
#else
  if (compiled) *compiled = 0;
#endif
  *sites = 0;
  *violations = 0;
  int (*readers[])(uint32_t*, uint64_t*, bool) = {check_read_classify, check_read_mr,
                                                   check_read_batched,  check_read_range,
                                                   check_read_window,   check_read_small};
  for (auto rd : readers) {
    uint32_t s = 0;
    uint64_t c = 0;
    int st = rd(&s, &c, reset != 0);
    if (st) return st;
    *sites |= s;
    *violations += c;
  }
  return ISPRIME_OK;
}

int isprime_measure_int_rates(int device, isprime_int_rates* out) {
  if (!out) return set_error(ISPRIME_EINVAL, "NULL argument");
  return measure_int_rates(device, out);
}

const char* isprime_strerror(int status) {
  switch (status) {
    case ISPRIME_OK: return "ok";
    case ISPRIME_EINVAL: return "invalid argument";
    case ISPRIME_ENOMEM: return "out of memory";
    case ISPRIME_ECUDA: return "CUDA error";
    case ISPRIME_EDOMAIN: return "input outside the domain (not an integer in [0, 2^53])";
    case ISPRIME_ETIMEDOUT: return "timed out";
    case ISPRIME_EBUSY: return "request exceeds the memory budget";
    default: return "unknown status";
  }
}

const char* isprime_last_error(void) { return t_last_error.c_str(); }

int isprime_version(void) { return 10000; }

}  // extern "C"
