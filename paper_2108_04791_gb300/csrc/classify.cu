// classify.cu -- load, classify, sieve lookup, trial division, enqueue.
//
// First stage of the array path (Sec. 6): every element is decided here
// unless it needs Miller-Rabin.
//   n < 2                   -> 0
//   n even                  -> n == 2
//   n < S (sieve limit)     -> one bit of the resident sieve (Sec. 6.1.3)
//   else trial division by the odd primes 3..p_k without division
//   (Sec. 6.1.2's input shrinking): a divisible n is composite (or equal to
//   the prime); a survivor below p_{k+1}^2 is prime; other survivors go to
//   the 32-bit (n < 2^32) or 64-bit Miller-Rabin queue, and their output byte
//   is written 0 here and set to 1 later if they are prime.
// Loads are 16-byte vector loads (two elements per thread, coalesced); queue
// appends are warp-aggregated (one atomic per warp and queue).
#include "arith.cuh"
#include "internal.h"
#include "tables.cuh"

namespace ip {

__constant__ TdTable c_td = make_td_table();

enum : int { kComposite = 0, kPrime = 1, kMR64 = 2, kMR32 = 3 };

__device__ __forceinline__ int classify_value(uint64_t n, const ClassifyArgs& a) {
  if (n < 2) return kComposite;
  if ((n & 1) == 0) return n == 2 ? kPrime : kComposite;
  if (n < a.sieve_limit)
    return (int)((__ldg(a.sieve + (n >> 6)) >> ((uint32_t)(n >> 1) & 31u)) & 1u);
  bool hit = false, equal = false;
  if (n < (1ull << 32)) {
    const uint32_t v = (uint32_t)n;
    for (uint32_t i = 0; i < a.ntd; ++i) {
      hit |= v * c_td.inv32[i] <= c_td.lim32[i];
      equal |= v == c_td.p[i];
    }
  } else {
#pragma unroll 4
    for (uint32_t i = 0; i < a.ntd; ++i) hit |= n * c_td.inv64[i] <= c_td.lim64[i];
  }
  if (equal) return kPrime;
  if (hit) return kComposite;
  if (n < a.td_square) return kPrime;
  return n < (1ull << 32) ? kMR32 : kMR64;
}

__device__ __forceinline__ void warp_push64(bool want, uint64_t v, uint32_t idx, uint64_t* qn,
                                            uint32_t* qi, uint32_t* counter) {
  const unsigned mask = __ballot_sync(0xFFFFFFFFu, want);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (want) {
    const uint32_t pos = base + __popc(mask & ((1u << lane) - 1u));
    qn[pos] = v;
    qi[pos] = idx;
  }
}

__device__ __forceinline__ void warp_push32(bool want, uint32_t v, uint32_t idx, uint32_t* qn,
                                            uint32_t* qi, uint32_t* counter) {
  const unsigned mask = __ballot_sync(0xFFFFFFFFu, want);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (want) {
    const uint32_t pos = base + __popc(mask & ((1u << lane) - 1u));
    qn[pos] = v;
    qi[pos] = idx;
  }
}

// Double input: finite, >= 0, integral and <= 2^53 (Sec. 8.1) converts
// exactly; anything else is invalid (output 0, counted).
__device__ __forceinline__ bool f64_to_u64(double x, uint64_t* v) {
  const bool ok = (x >= 0.0) && (x <= 9007199254740992.0) && (floor(x) == x);
  *v = ok ? (uint64_t)x : 0ull;
  return ok;
}

template <typename T>
struct Loader;

template <>
struct Loader<uint64_t> {
  static __device__ __forceinline__ void pair(const void* p, uint64_t i, uint64_t* v0, uint64_t* v1,
                                              bool* ok0, bool* ok1) {
    const uint4 q = __ldcs(reinterpret_cast<const uint4*>(static_cast<const uint64_t*>(p) + i));
    *v0 = ((uint64_t)q.y << 32) | q.x;
    *v1 = ((uint64_t)q.w << 32) | q.z;
    *ok0 = *ok1 = true;
  }
  static __device__ __forceinline__ uint64_t one(const void* p, uint64_t i, bool* ok) {
    *ok = true;
    return static_cast<const uint64_t*>(p)[i];
  }
};

template <>
struct Loader<double> {
  static __device__ __forceinline__ void pair(const void* p, uint64_t i, uint64_t* v0, uint64_t* v1,
                                              bool* ok0, bool* ok1) {
    const double2 q = __ldcs(reinterpret_cast<const double2*>(static_cast<const double*>(p) + i));
    *ok0 = f64_to_u64(q.x, v0);
    *ok1 = f64_to_u64(q.y, v1);
  }
  static __device__ __forceinline__ uint64_t one(const void* p, uint64_t i, bool* ok) {
    uint64_t v;
    *ok = f64_to_u64(static_cast<const double*>(p)[i], &v);
    return v;
  }
};

// Handles one element outside the vectorised loop (alignment head / tail).
template <typename T>
__device__ void classify_single(const ClassifyArgs& a, uint64_t i) {
  bool ok;
  const uint64_t v = Loader<T>::one(a.in, i, &ok);
  int d = ok ? classify_value(v, a) : kComposite;
  if (!ok && a.invalid) atomicAdd(a.invalid, 1ull);
  a.out[i] = (uint8_t)(d == kPrime);
  if (d == kMR64) {
    const uint32_t pos = atomicAdd(&a.counters[0], 1u);
    a.q64_n[pos] = v;
    a.q64_idx[pos] = (uint32_t)i;
  } else if (d == kMR32) {
    const uint32_t pos = atomicAdd(&a.counters[1], 1u);
    a.q32_n[pos] = (uint32_t)v;
    a.q32_idx[pos] = (uint32_t)i;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) classify_kernel(ClassifyArgs a) {
  const int lane = threadIdx.x & 31;
  const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t head = a.head;
  const uint64_t npairs = (a.n - head) / 2;
  // Vectorised body: pair p covers elements head + 2p and head + 2p + 1.
  // The loop bound is per warp, so every lane takes part in the ballots.
  for (uint64_t wbase = (gtid & ~31ull); wbase < npairs; wbase += nthreads) {
    const uint64_t p = wbase + lane;
    const bool valid = p < npairs;
    uint64_t v0 = 0, v1 = 0;
    bool ok0 = true, ok1 = true;
    int d0 = kComposite, d1 = kComposite;
    const uint64_t i0 = head + 2 * p;
    if (valid) {
      Loader<T>::pair(a.in, i0, &v0, &v1, &ok0, &ok1);
      d0 = ok0 ? classify_value(v0, a) : kComposite;
      d1 = ok1 ? classify_value(v1, a) : kComposite;
      const uint8_t o0 = (uint8_t)(d0 == kPrime), o1 = (uint8_t)(d1 == kPrime);
      if (a.pair_store)
        *reinterpret_cast<uint16_t*>(a.out + i0) = (uint16_t)(o0 | (o1 << 8));
      else {
        a.out[i0] = o0;
        a.out[i0 + 1] = o1;
      }
    }
    if (a.invalid) {
      const unsigned bad = __ballot_sync(0xFFFFFFFFu, valid && !ok0) ;
      const unsigned bad1 = __ballot_sync(0xFFFFFFFFu, valid && !ok1);
      if (lane == 0 && (bad | bad1))
        atomicAdd(a.invalid, (unsigned long long)(__popc(bad) + __popc(bad1)));
    }
    warp_push64(d0 == kMR64, v0, (uint32_t)i0, a.q64_n, a.q64_idx, &a.counters[0]);
    warp_push64(d1 == kMR64, v1, (uint32_t)(i0 + 1), a.q64_n, a.q64_idx, &a.counters[0]);
    warp_push32(d0 == kMR32, (uint32_t)v0, (uint32_t)i0, a.q32_n, a.q32_idx, &a.counters[1]);
    warp_push32(d1 == kMR32, (uint32_t)v1, (uint32_t)(i0 + 1), a.q32_n, a.q32_idx, &a.counters[1]);
  }
  // Alignment head (at most one element) and odd tail (at most one).
  if (gtid == 0) {
    for (uint64_t i = 0; i < head; ++i) classify_single<T>(a, i);
    for (uint64_t i = head + 2 * npairs; i < a.n; ++i) classify_single<T>(a, i);
  }
}

template <typename T>
static int launch_classify(isprime_ctx* ctx, const ClassifyArgs& a, cudaStream_t s, int kid,
                           const char* name) {
  const uint32_t block = ctx->tune.classify_block;
  const uint64_t npairs = (a.n - a.head) / 2;
  uint64_t want = (npairs + block - 1) / block;
  const uint64_t cap = (uint64_t)ctx->sm_count * ctx->tune.blocks_per_sm;
  unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  TimedLaunch tl;
  int st = launch_begin(ctx, kid, s, &tl);
  if (st) return st;
  classify_kernel<T><<<grid, block, 0, s>>>(a);
  return launch_end(ctx, s, &tl, name);
}

int launch_classify_u64(isprime_ctx* ctx, const ClassifyArgs& a, cudaStream_t s) {
  return launch_classify<uint64_t>(ctx, a, s, ISPRIME_K_CLASSIFY_U64, "classify_kernel<u64>");
}

int launch_classify_f64(isprime_ctx* ctx, const ClassifyArgs& a, cudaStream_t s) {
  return launch_classify<double>(ctx, a, s, ISPRIME_K_CLASSIFY_F64, "classify_kernel<f64>");
}

// Launch without a context (explicit grid and block); used by the
// allocation-free entry point.
int launch_classify_u64_raw(const ClassifyArgs& a, unsigned grid, unsigned block, cudaStream_t s) {
  classify_kernel<uint64_t><<<grid, block, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ISPRIME_OK : cuda_fail(e, "classify_kernel<u64>");
}

uint64_t td_square_for(uint32_t ntd) {
  const uint64_t next = ntd < (uint32_t)kMaxTdPrimes ? kTdPrimeList[ntd] : kTdNextPrimeAfterList;
  return next * next;
}

}  // namespace ip
