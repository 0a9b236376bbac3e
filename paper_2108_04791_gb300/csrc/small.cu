// small.cu -- the latency path for scalars and tiny arrays.
//
// The paper answers a scalar according to its size class (Sec. 1): Miller-
// Rabin with Eq. 4's bases for large values (Sec. 2), wheel trial division
// for medium ones (Sec. 3), odd trial division for small ones (Sec. 4);
// Table 4 reports the time of one call per bit size.  On the GPU the time of
// one call is launch latency plus the longest dependent chain of one value's
// test, so this path gives each value a whole warp and splits its test over
// the lanes:
//   * below the sieve limit S: one lookup in the resident bitmap;
//   * trial division by the 53 odd primes 3..251, lane l testing the l-th and
//     (l+32)-th prime, decided by one vote; a survivor below 257^2 is prime;
//   * below 2^32 (contexts with S < 2^32): bases 2, 7, 61 on lanes 0-2;
//   * otherwise the seven bases of Eq. 4 on lanes 0-6 at the same time.
// Each lane computes a^d right to left: the squarings of the base and the
// multiplications into the result are two independent chains, so the
// dependent chain is bitlen(d) - 1 squarings.  One launch, no queues and no
// scratch, so these calls need no ordering against the context's other work.
//
// Host arrays of at most kInlineMax values travel inside the kernel's
// parameters (no host-to-device copy) and the results are written straight
// into mapped pinned host memory (no device-to-host copy): a call is one
// launch and one synchronisation.
#include <string.h>

#include "device_common.cuh"
#include "internal.h"

namespace ip {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSmallBlock = 128;  // four warps, one value each per step

// x = a^d in Montgomery form for odd d >= 1 and aR = a R mod n, right to left.
__device__ __forceinline__ uint64_t pow_right_to_left(const Mont64& M, uint64_t aR, uint64_t d) {
  using Ops = MontOps<0>;
  uint64_t x = aR, p = aR;  // bit 0 of d is set
  for (d >>= 1; d; d >>= 1) {
    p = Ops::sqr(p, M);
    if (d & 1) x = Ops::mul(x, p, M);
  }
  return x;
}

// isprime(n) decided by one whole warp; every lane passes the same n and
// every lane gets the answer.
__device__ __forceinline__ bool warp_isprime(uint64_t n, const uint32_t* sieve, uint64_t S,
                                             int lane) {
  if (n < 2) return false;
  if ((n & 1) == 0) return n == 2;
  if (n < S) return (__ldg(sieve + (n >> 6)) >> ((uint32_t)(n >> 1) & 31u)) & 1u;
  bool hit = false, equal = false;
  for (int i = lane; i < kMaxTdPrimes; i += 32) {
    hit |= n * c_td.inv64[i] <= c_td.lim64[i];
    equal |= n == c_td.p[i];
  }
  if (__any_sync(kFull, equal)) return true;
  if (__any_sync(kFull, hit)) return false;
  if (n < (uint64_t)kTdNextPrimeAfterList * kTdNextPrimeAfterList) return true;
  bool pass = true;
  if (n < (1ull << 32)) {
    if (lane < kNumBases32) {
      const Mont32 M = mont32_setup((uint32_t)n);
      uint32_t d = (uint32_t)n - 1;
      const int s = ctz32(d);
      d >>= s;
      pass = sprp32(M, c_bases.b32[lane], d, s);  // every base < 257^2 <= n
    }
  } else if (lane < kNumBases64) {
    const Mont64 M = mont64_setup(n);
    const uint64_t r2 = mont64_r2<0>(M);
    uint64_t d = n - 1;
    const int s = ctz64(d);
    d >>= s;
    const uint64_t aR = MontOps<0>::mul((uint64_t)c_bases.b64[lane], r2, M);  // bases < 2^32 <= n
    pass = sprp_tail64<0>(M, pow_right_to_left(M, aR, d), s);
  }
  return __all_sync(kFull, pass);
}

template <typename T>
__device__ __forceinline__ bool load_value(const T* in, uint64_t i, uint64_t* v);
template <>
__device__ __forceinline__ bool load_value<uint64_t>(const uint64_t* in, uint64_t i, uint64_t* v) {
  *v = __ldg(in + i);
  return true;
}
template <>
__device__ __forceinline__ bool load_value<double>(const double* in, uint64_t i, uint64_t* v) {
  return f64_to_u64(__ldg(in + i), v);
}

// One warp per element, grid-stride over warps.
template <typename T>
__global__ void __launch_bounds__(kSmallBlock) small_kernel(const T* __restrict__ in,
                                                            uint8_t* __restrict__ out, uint64_t n,
                                                            const uint32_t* __restrict__ sieve,
                                                            uint64_t S,
                                                            unsigned long long* invalid,
                                                            unsigned long long* invalid_ctx) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t bad = 0;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    uint64_t v;
    const bool ok = load_value<T>(in, i, &v);  // the same for the whole warp
    const bool prime = ok && warp_isprime(v, sieve, S, lane);
    if (lane == 0) {
      out[i] = prime ? 1 : 0;
      bad += ok ? 0 : 1;
    }
  }
  if (lane == 0 && bad) {
    if (invalid) atomicAdd(invalid, (unsigned long long)bad);
    if (invalid_ctx) atomicAdd(invalid_ctx, (unsigned long long)bad);
  }
}

template <int kCap>
struct InlineValues {
  uint64_t v[kCap];
};

// Values from the kernel parameters, bytes to mapped host memory.
template <int kCap>
__global__ void __launch_bounds__(kSmallBlock)
    inline_kernel(const __grid_constant__ InlineValues<kCap> iv, uint32_t n,
                  uint8_t* __restrict__ out, const uint32_t* __restrict__ sieve, uint64_t S) {
  const int lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
    const bool prime = warp_isprime(iv.v[i], sieve, S, lane);
    if (lane == 0) out[i] = prime ? 1 : 0;
  }
}

unsigned small_grid(const isprime_ctx* ctx, uint64_t n) {
  const uint64_t warps_per_block = kSmallBlock / 32;
  const uint64_t want = (n + warps_per_block - 1) / warps_per_block;
  const uint64_t cap = (uint64_t)ctx->sm_count * (2048 / kSmallBlock);
  return (unsigned)(want < cap ? want : cap);
}

template <int kCap>
int launch_inline(isprime_ctx* ctx, const uint64_t* h_in, uint32_t n, cudaStream_t s) {
  InlineValues<kCap> iv;
  memcpy(iv.v, h_in, (size_t)n * sizeof(uint64_t));
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_SMALL, s, &tl);
  if (st) return st;
  const unsigned block = n < kSmallBlock / 32 ? 32u * n : kSmallBlock;
  inline_kernel<kCap><<<small_grid(ctx, n), block, 0, s>>>(iv, n, ctx->d_inline_out, ctx->d_sieve,
                                                           sieve_cut(ctx));
  return launch_end(ctx, s, &tl, "inline_kernel");
}

}  // namespace

IP_CHECK_READER(check_read_small)

int launch_small_u64(isprime_ctx* ctx, const uint64_t* d_in, uint8_t* d_out, size_t n,
                     cudaStream_t s) {
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_SMALL, s, &tl);
  if (st) return st;
  small_kernel<uint64_t><<<small_grid(ctx, n), kSmallBlock, 0, s>>>(d_in, d_out, n, ctx->d_sieve,
                                                                    sieve_cut(ctx), nullptr, nullptr);
  return launch_end(ctx, s, &tl, "small_kernel<u64>");
}

int launch_small_f64(isprime_ctx* ctx, const double* d_in, uint8_t* d_out, size_t n,
                     unsigned long long* d_invalid, unsigned long long* d_invalid_ctx,
                     cudaStream_t s) {
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_SMALL, s, &tl);
  if (st) return st;
  small_kernel<double><<<small_grid(ctx, n), kSmallBlock, 0, s>>>(d_in, d_out, n, ctx->d_sieve,
                                                                  sieve_cut(ctx), d_invalid,
                                                                  d_invalid_ctx);
  return launch_end(ctx, s, &tl, "small_kernel<f64>");
}

// Host values in, host bytes out, n <= kInlineMax.  The mapped result
// buffer belongs to the context: inline_mu serialises its users.
int inline_run(isprime_ctx* ctx, const uint64_t* h_in, uint8_t* h_out, size_t n, cudaStream_t s) {
  std::lock_guard<std::mutex> inline_lock(ctx->inline_mu);
  if (!ctx->h_inline_out) {
    void* h = nullptr;
    IP_CUDA(cudaHostAlloc(&h, kInlineMax, cudaHostAllocMapped));
    ctx->h_inline_out = static_cast<uint8_t*>(h);
    void* d = nullptr;
    IP_CUDA(cudaHostGetDevicePointer(&d, h, 0));
    ctx->d_inline_out = static_cast<uint8_t*>(d);
  }
  const uint32_t m = (uint32_t)n;
  {
    std::lock_guard<std::mutex> lock(ctx->mu);  // timing records and counters
    int st = m == 1 ? launch_inline<1>(ctx, h_in, m, s)
                    : m <= 32 ? launch_inline<32>(ctx, h_in, m, s)
                              : launch_inline<kInlineMax>(ctx, h_in, m, s);
    if (st) return st;
    ctx->stats.calls++;
    ctx->stats.elements += n;
  }
  IP_CUDA(cudaStreamSynchronize(s));
  memcpy(h_out, ctx->h_inline_out, n);
  return ISPRIME_OK;
}

}  // namespace ip

namespace ip {

namespace {

// Element e of a batch whose descriptors hold element prefix sums in
// tile_begin: the array is the last one whose prefix is <= e, found by a
// 32-way search with one probe per lane per round (ceil(log32(arrays))
// rounds; every lane of the warp holds the same e).
__device__ __forceinline__ uint32_t find_array(const BatchDesc* __restrict__ descs,
                                               uint32_t n_arrays, uint64_t e, int lane) {
  uint32_t lo = 0, hi = n_arrays;  // answer in [lo, hi), prefix(lo) <= e
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t idx = lo + (uint32_t)lane * step;
    const bool ok = idx < hi && __ldg(&descs[idx].tile_begin) <= e;
    const unsigned m = __ballot_sync(kFull, ok);  // lanes 0..k-1 set, lane 0 always
    const uint32_t last = 31u - (uint32_t)__clz((int)m);
    lo = lo + last * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

__global__ void __launch_bounds__(kSmallBlock)
    small_batched_kernel(const BatchDesc* __restrict__ descs, uint32_t n_arrays, uint64_t total,
                         const uint32_t* __restrict__ sieve, uint64_t S) {
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t e = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += nwarps) {
    const uint32_t a = find_array(descs, n_arrays, e, lane);
    const uint64_t j = e - descs[a].tile_begin;
    // a plain load: the array may be mapped host memory (the server's short requests)
    const bool prime = warp_isprime(descs[a].in[j], sieve, S, lane);
    if (lane == 0 && IP_CHECK(j < descs[a].n, kChkSmallOut)) descs[a].out[j] = prime ? 1 : 0;
  }
}

}  // namespace

int launch_small_batched(isprime_ctx* ctx, const BatchDesc* d_descs, uint32_t n_arrays,
                         uint64_t total, cudaStream_t s) {
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_SMALL, s, &tl);
  if (st) return st;
  small_batched_kernel<<<small_grid(ctx, total), kSmallBlock, 0, s>>>(d_descs, n_arrays, total,
                                                                      ctx->d_sieve, sieve_cut(ctx));
  return launch_end(ctx, s, &tl, "small_batched_kernel");
}

}  // namespace ip
