// window.cu -- the per-call path choice between the queue path and a sieve
// of the array's value window (the GPU analogue of Sec. 6.2, Eqs. 7-8).
//
// The paper chooses per call between trial division up to sqrt(max) and a
// sieve of every integer up to max(N) followed by a membership search,
// from the array's length and maximum (two linear fits).  Here every value
// below the resident sieve limit S is already one bit lookup, so the choice
// only matters above S, where it is between
//   the queue path   classify + trial division + Miller-Rabin per element
//                    (cost ~ N), and
//   the window path  sieve every integer of [min, max] with the range kernels
//                    (isprime_range: a shared-memory sieve by the primes below
//                    2^16, Miller-Rabin on its survivors) into a byte per
//                    integer, then out[i] = window[in[i] - min] (cost ~ W,
//                    W = max - min + 1, plus a gather of N bytes).
// The window path wins when the array is dense in its window (W small next
// to N: shuffled windows of consecutive values, values with repeats).  The
// rule: take it when max >= S, W <= kWindowMax and 16 W <= ratio16 N, where
// ratio16 (tuning window_ratio16, 0 = never) is fitted on this GPU by the
// autotuner.  Deciding needs the array's min and max on the host, so a call
// that considers the window path runs one reduction kernel and waits for it
// (the call is then synchronous up to that point).
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace ip {

constexpr uint64_t kWindowMax = (uint64_t)1 << 30;  // bytes of the window buffer at most

// Min and max of n values: a grid-stride pass, a warp and block reduction,
// one atomicMin / atomicMax per block into mm[0] / mm[1] (preset to ~0 / 0).
__global__ void __launch_bounds__(256) minmax_kernel(const uint64_t* __restrict__ in, uint64_t n,
                                                     unsigned long long* mm) {
  __shared__ unsigned long long s_lo[8], s_hi[8];
  uint64_t lo = ~0ull, hi = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = __ldcs(in + i);
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t l = __shfl_xor_sync(0xFFFFFFFFu, lo, o), h = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
    lo = l < lo ? l : lo;
    hi = h > hi ? h : hi;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = s_lo[w] < lo ? s_lo[w] : lo;
      hi = s_hi[w] > hi ? s_hi[w] : hi;
    }
    atomicMin(&mm[0], (unsigned long long)lo);
    atomicMax(&mm[1], (unsigned long long)hi);
  }
}

// out[i] = win[in[i] - lo] for i < n; every in[i] lies in [lo, lo + W).
__global__ void __launch_bounds__(256) window_gather_kernel(const uint64_t* __restrict__ in,
                                                            uint8_t* __restrict__ out, uint64_t n,
                                                            const uint8_t* __restrict__ win,
                                                            uint64_t lo, uint64_t w) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = __ldcs(in + i) - lo;
    if (IP_CHECK(k < w, kChkWindow)) out[i] = win[k];
  }
}

IP_CHECK_READER(check_read_window)

// Min and max of a device array (synchronous on s).
int array_minmax(isprime_ctx* ctx, const uint64_t* d_in, size_t n, cudaStream_t s, uint64_t* lo,
                 uint64_t* hi) {
  if (!ctx->d_mm) {
    IP_CUDA(cudaMalloc(&ctx->d_mm, 2 * sizeof(unsigned long long)));
    IP_CUDA(cudaMallocHost(&ctx->h_mm, 2 * sizeof(unsigned long long)));
  }
  IP_CUDA(cudaMemsetAsync(ctx->d_mm, 0xFF, sizeof(unsigned long long), s));
  IP_CUDA(cudaMemsetAsync(ctx->d_mm + 1, 0, sizeof(unsigned long long), s));
  const uint64_t want = (n + 255) / 256;
  const uint64_t cap = (uint64_t)ctx->sm_count * 8;
  minmax_kernel<<<(unsigned)std::max<uint64_t>(1, std::min(want, cap)), 256, 0, s>>>(d_in, n,
                                                                                     ctx->d_mm);
  IP_CUDA(cudaGetLastError());
  IP_CUDA(cudaMemcpyAsync(ctx->h_mm, ctx->d_mm, 2 * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, s));
  IP_CUDA(cudaStreamSynchronize(s));
  *lo = ctx->h_mm[0];
  *hi = ctx->h_mm[1];
  return ISPRIME_OK;
}

// v[i] = lo + (i a mod w) for i < n, w a power of two and a odd: every
// integer of the window [lo, lo + w) equally often (n >= w) or n distinct
// ones (n <= w).
__global__ void window_fill_kernel(uint64_t* v, uint64_t n, uint64_t lo, uint64_t w, uint64_t a) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = lo + ((i * a) & (w - 1));
}

// Fits the crossover of the window path on this GPU for arrays of about n
// values near `near` (autotuner).  On m values (n rounded down to a power of
// two in [2^16, 2^24]) spread over windows of m/4 and of m integers
// (densities 4 and 1), times the queue path and the window path; with the
// window path's time linear in the window width W, t_win(W) = alpha + beta W,
// it wins for W < W* = (t_queue - alpha) / beta, so ratio16 = 16 W* / m (0
// when W* <= 0: the fixed cost alone exceeds the queue path's time).  The
// context's tuning is left as it was.
int window_fit(isprime_ctx* ctx, uint64_t near, size_t n, cudaStream_t s, uint32_t* ratio16) {
  *ratio16 = 0;
  size_t m = (size_t)1 << 16;
  while (m * 2 <= n && m * 2 <= ((size_t)1 << 24)) m *= 2;
  uint64_t lo = near > (uint64_t)m ? near - (uint64_t)m : 0;
  const uint64_t cut = sieve_cut(ctx);
  if (lo < cut) lo = cut;
  if (lo > UINT64_MAX - (uint64_t)m) lo = UINT64_MAX - (uint64_t)m;
  uint64_t* d_v = nullptr;
  uint8_t* d_o = nullptr;
  IP_CUDA(cudaMalloc(&d_v, m * sizeof(uint64_t)));
  cudaError_t e = cudaMalloc(&d_o, m);
  if (e != cudaSuccess) {
    cudaFree(d_v);
    return cuda_fail(e, "cudaMalloc (window fit)");
  }
  const isprime_tuning saved = ctx->tune;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](uint64_t w, uint32_t r16, float* best) -> int {
    window_fill_kernel<<<(unsigned)std::min<uint64_t>((m + 255) / 256, 1024), 256, 0, s>>>(
        d_v, m, lo, w, 0x9E3779B97F4A7C15ull);
    IP_CUDA(cudaGetLastError());
    isprime_tuning t = saved;
    t.window_ratio16 = r16;
    t.small_max = 0;
    int st = isprime_ctx_set_tuning(ctx, &t);
    if (st) return st;
    *best = 1e30f;
    for (int r = 0; r < 4; ++r) {
      IP_CUDA(cudaEventRecord(e0, s));
      if ((st = isprime_u64_ctx(ctx, d_v, d_o, m, (isprime_stream)s))) return st;
      IP_CUDA(cudaEventRecord(e1, s));
      IP_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      IP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0) *best = std::min(*best, ms);
    }
    return ISPRIME_OK;
  };
  float tq = 0, tw1 = 0, tw4 = 0;  // tw1: W = m / 4, tw4: W = m
  int st = timed((uint64_t)m, 0, &tq);
  if (!st) st = timed((uint64_t)m / 4, 4096, &tw1);
  if (!st) st = timed((uint64_t)m, 4096, &tw4);
  isprime_ctx_set_tuning(ctx, &saved);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_v);
  cudaFree(d_o);
  if (st) return st;
  const double beta = (double)(tw4 - tw1) / (0.75 * (double)m);  // ms per window integer
  const double alpha = (double)tw1 - beta * 0.25 * (double)m;
  if (beta <= 0 || alpha >= (double)tq) return ISPRIME_OK;
  const double r = 16.0 * ((double)tq - alpha) / (beta * (double)m);
  *ratio16 = (uint32_t)std::min(4096.0, std::max(0.0, r));
  ctx->fitted_window_ratio16 = *ratio16;
  return ISPRIME_OK;
}

// Decides the path of one u64 call and, when it is the window path, runs it
// on stream s (*taken = true).  The caller holds ctx->mu and has ordered s
// after the context's previous use of its queues.
int window_try(isprime_ctx* ctx, const uint64_t* d_in, uint8_t* d_out, size_t n, cudaStream_t s,
               bool* taken) {
  *taken = false;
  const uint32_t ratio16 = ctx->tune.window_ratio16;
  if (ratio16 == 0 || n < ((size_t)1 << 16)) return ISPRIME_OK;
  uint64_t lo = 0, hi = 0;
  int st = array_minmax(ctx, d_in, n, s, &lo, &hi);
  if (st) return st;
  ctx->last_window_lo = lo;
  ctx->last_window_hi = hi;
  if (hi < sieve_cut(ctx)) return ISPRIME_OK;  // every value is a bit lookup already
  const uint64_t w_minus1 = hi - lo;           // W - 1 (W may be 2^64)
  if (w_minus1 >= kWindowMax) return ISPRIME_OK;
  const uint64_t w = w_minus1 + 1;
  if ((unsigned __int128)w * 16 > (unsigned __int128)n * ratio16) return ISPRIME_OK;
  if (ctx->window_cap < w) {
    cudaFree(ctx->d_window);
    ctx->d_window = nullptr;
    ctx->window_cap = 0;
    const size_t bytes = std::max<size_t>((size_t)w, (size_t)1 << 20);
    IP_CUDA(cudaMalloc(&ctx->d_window, bytes));
    ctx->window_cap = bytes;
  }
  if ((st = range_run(ctx, lo, w, ctx->d_window, s))) return st;
  const uint64_t want = (n + 255) / 256;
  TimedLaunch tl;
  if ((st = launch_begin(ctx, ISPRIME_K_RANGE, s, &tl))) return st;
  const uint64_t gcap = (uint64_t)ctx->sm_count * 16;
  window_gather_kernel<<<(unsigned)std::min(want, gcap), 256, 0, s>>>(d_in, d_out, n,
                                                                        ctx->d_window, lo, w);
  if ((st = launch_end(ctx, s, &tl, "window_gather_kernel"))) return st;
  ctx->stats.window_calls++;
  *taken = true;
  return ISPRIME_OK;
}

}  // namespace ip
