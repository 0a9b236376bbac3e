// mr.cu -- deterministic Miller-Rabin on the compacted survivor queues.
//
// Sec. 2.1: n - 1 = 2^s d with d odd; n passes base a when a^d = 1 or
// a^(2^r d) = n - 1 for some r < s (the textbook strong condition; the
// printed "+-1" of Eq. 1 is read this way).  The seven bases of Eq. 4 decide
// every n < 2^64; {2, 7, 61} decide every n < 4,759,123,141.
//
// Kernels (each a grid-stride loop over a queue whose length is read on the
// device, so no host synchronisation separates the stages):
//   mr64_base2_kernel  base 2 for every 64-bit survivor of trial division;
//                      "multiply by 2" is a modular doubling.  Passing
//                      elements (the primes and rare strong pseudoprimes) are
//                      compacted with warp ballots into a second queue, so
//                      the next kernel runs on dense warps of likely primes
//                      instead of idling behind early-exiting composites.
//   mr64_rest_kernel   the six remaining bases, 4-bit fixed-window
//                      exponentiation with the per-thread window table in
//                      shared memory; writes 1 for primes.
//   mr32_kernel        bases 2, 7, 61 in 32-bit Montgomery arithmetic for
//                      survivors in [S, 2^32) (only when S < 2^32).
// All arithmetic is in arith.cuh (ModExp / ModMultiply / ModAdd of
// Sec. 2.2-2.4 as Montgomery multiplication and doubling).
#include "arith.cuh"
#include "internal.h"
#include "tables.cuh"

namespace ip {

__constant__ BaseTable c_bases = make_base_table();

constexpr int kWin = 4;
constexpr int kTab = 1 << kWin;

__global__ void __launch_bounds__(256) mr64_base2_kernel(const uint64_t* __restrict__ qn,
                                                         uint32_t* __restrict__ counters,
                                                         uint32_t* __restrict__ q64b) {
  const uint32_t count = *(volatile uint32_t*)&counters[0];
  const int lane = threadIdx.x & 31;
  const uint32_t gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  for (uint32_t wbase = gtid & ~31u; wbase < count; wbase += nthreads) {
    const uint32_t i = wbase + lane;
    bool pass = false;
    if (i < count) {
      const uint64_t n = qn[i];
      const Mont64 M = mont64_setup(n);
      uint64_t d = n - 1;
      const int s = ctz64(d);
      d >>= s;
      pass = sprp2_64(M, d, s);
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, pass);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&counters[2], (uint32_t)__popc(mask));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (pass) q64b[base + __popc(mask & ((1u << lane) - 1u))] = i;
    }
  }
}

// a^d mod n in Montgomery form by 4-bit fixed windows over the nibbles of d.
// tab points at this thread's column of the shared table (stride `ld`).
__device__ __forceinline__ uint64_t mont_pow_win4(const Mont64& M, uint64_t aR, uint64_t d,
                                                  uint64_t* tab, int ld) {
  const uint64_t n = M.n, ninv = M.ninv;
  tab[0] = M.one;
  tab[ld] = aR;
  uint64_t t = mont_sqr(aR, n, ninv);
  tab[2 * ld] = t;
#pragma unroll
  for (int j = 3; j < kTab; ++j) {
    t = mont_mul(t, aR, n, ninv);
    tab[j * ld] = t;
  }
  const int nib = (64 - clz64(d) + kWin - 1) / kWin;  // nibbles in d (d >= 1)
  uint64_t x = tab[(int)((d >> (kWin * (nib - 1))) & (kTab - 1)) * ld];
  for (int k = nib - 2; k >= 0; --k) {
#pragma unroll
    for (int q = 0; q < kWin; ++q) x = mont_sqr(x, n, ninv);
    x = mont_mul(x, tab[(int)((d >> (kWin * k)) & (kTab - 1)) * ld], n, ninv);
  }
  return x;
}

__global__ void __launch_bounds__(256) mr64_rest_kernel(const uint64_t* __restrict__ qn,
                                                        const uint32_t* __restrict__ qidx,
                                                        const uint32_t* __restrict__ q64b,
                                                        const uint32_t* __restrict__ counters,
                                                        uint8_t* __restrict__ out) {
  extern __shared__ uint64_t s_tab[];  // kTab x blockDim
  uint64_t* tab = s_tab + threadIdx.x;
  const int ld = blockDim.x;
  const uint32_t count = *(volatile const uint32_t*)&counters[2];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint32_t j = q64b[i];
    const uint64_t n = qn[j];
    const Mont64 M = mont64_setup(n);
    const uint64_t r2 = mont64_r2(M);
    uint64_t d = n - 1;
    const int s = ctz64(d);
    d >>= s;
    bool prime = true;
    // n >= 2^32 > every base, so no base is 0 mod n.
#pragma unroll 1
    for (int b = 1; b < kNumBases64; ++b) {
      const uint64_t aR = mont_mul((uint64_t)c_bases.b64[b], r2, n, M.ninv);
      const uint64_t x = mont_pow_win4(M, aR, d, tab, ld);
      if (!sprp_tail64(M, x, s)) {
        prime = false;
        break;
      }
    }
    if (prime) out[qidx[j]] = 1;
  }
}

__global__ void __launch_bounds__(256) mr32_kernel(const uint32_t* __restrict__ qn,
                                                   const uint32_t* __restrict__ qidx,
                                                   const uint32_t* __restrict__ counters,
                                                   uint8_t* __restrict__ out) {
  const uint32_t count = *(volatile const uint32_t*)&counters[1];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const uint32_t n = qn[i];
    const Mont32 M = mont32_setup(n);
    uint32_t d = n - 1;
    const int s = ctz32(d);
    d >>= s;
    bool prime = true;
#pragma unroll 1
    for (int b = 0; b < kNumBases32; ++b) {
      const uint32_t a = c_bases.b32[b] % n;
      if (a == 0) continue;  // base divisible by n: skipped (n is 7 or 61 here)
      if (!sprp32(M, a, d, s)) {
        prime = false;
        break;
      }
    }
    if (prime) out[qidx[i]] = 1;
  }
}

int launch_mr(isprime_ctx* ctx, uint8_t* out, cudaStream_t s) {
  const uint32_t block = ctx->tune.mr_block;
  const unsigned grid = (unsigned)ctx->sm_count * ctx->tune.blocks_per_sm;
  TimedLaunch tl;
  int st;
  if (ctx->sieve_limit < (1ull << 32)) {
    if ((st = launch_begin(ctx, ISPRIME_K_MR32, s, &tl))) return st;
    mr32_kernel<<<grid, block, 0, s>>>(ctx->q.q32_n, ctx->q.q32_idx, ctx->q.counters, out);
    if ((st = launch_end(ctx, s, &tl, "mr32_kernel"))) return st;
  }
  if ((st = launch_begin(ctx, ISPRIME_K_MR64_BASE2, s, &tl))) return st;
  mr64_base2_kernel<<<grid, block, 0, s>>>(ctx->q.q64_n, ctx->q.counters, ctx->q.q64b);
  if ((st = launch_end(ctx, s, &tl, "mr64_base2_kernel"))) return st;
  if ((st = launch_begin(ctx, ISPRIME_K_MR64_REST, s, &tl))) return st;
  const size_t smem = (size_t)kTab * block * sizeof(uint64_t);
  mr64_rest_kernel<<<grid, block, smem, s>>>(ctx->q.q64_n, ctx->q.q64_idx, ctx->q.q64b,
                                              ctx->q.counters, out);
  return launch_end(ctx, s, &tl, "mr64_rest_kernel");
}

// Launch without a context (explicit grid and block and queue pointers);
// used by the allocation-free entry point.
int launch_mr_raw(const Queues& q, uint8_t* out, bool with_mr32, unsigned grid, unsigned block,
                  cudaStream_t s) {
  if (with_mr32) mr32_kernel<<<grid, block, 0, s>>>(q.q32_n, q.q32_idx, q.counters, out);
  mr64_base2_kernel<<<grid, block, 0, s>>>(q.q64_n, q.counters, q.q64b);
  const size_t smem = (size_t)kTab * block * sizeof(uint64_t);
  mr64_rest_kernel<<<grid, block, smem, s>>>(q.q64_n, q.q64_idx, q.q64b, q.counters, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ISPRIME_OK : cuda_fail(e, "Miller-Rabin kernels");
}

}  // namespace ip
