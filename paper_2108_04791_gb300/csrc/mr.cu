// mr.cu -- deterministic Miller-Rabin on the compacted survivor queues.
//
// Sec. 2.1: n - 1 = 2^s d with d odd; n passes base a when a^d = 1 or
// a^(2^r d) = n - 1 for some r < s (the textbook strong condition; the
// printed "+-1" of Eq. 1 is read this way).  The seven bases of Eq. 4 decide
// every n < 2^64; {2, 7, 61} decide every n < 4,759,123,141.
//
// Kernels (each a grid-stride loop over a queue whose length is read on the
// device, so no host synchronisation separates the stages):
//   mr64_base2_kernel  base 2 for every 64-bit survivor of trial division, by
//                      4-bit windows where "multiply by 2^w" is x 2^w - q n
//                      with an estimated quotient (base2_window 1), or a
//                      Montgomery product with the table 2^w R (4), or
//                      binary with a modular doubling per set bit (0).  Passing elements (the primes and rare
//                      strong pseudoprimes) are compacted with warp ballots
//                      into a second queue, so the next kernel runs on dense
//                      warps of likely primes instead of idling behind
//                      early-exiting composites.  With the compaction threshold
//                      compact_min <= 32, a warp left with at least that many
//                      survivors finishes them itself.
//   mr64_rest_kernel   the six remaining bases, 4-bit fixed-window
//                      exponentiation with the per-thread window table in
//                      shared memory.  On chunks of at most 2^22 elements a
//                      queue shorter than the grid is spread over 6, 3 or 2
//                      threads per survivor (the base-2 kernel then marks its
//                      survivors prime and a failing base clears the byte);
//                      otherwise one survivor per thread, writing 1 for primes.
//   mr32_kernel        bases 2, 7, 61 in 32-bit Montgomery arithmetic for
//                      survivors between the sieve cutover and 2^32.
// All arithmetic is in arith.cuh (ModExp / ModMultiply / ModAdd of
// Sec. 2.2-2.4 as Montgomery multiplication and doubling).
#include "device_common.cuh"
#include "internal.h"

namespace ip {

// kMode: the base-2 schedule (the tuning field base2_window): 0 binary with
// a modular doubling per set bit, 1 4-bit windows with x 2^w mod n by a
// quotient estimate, 4 4-bit windows with the table 2^w R in shared memory.
// kRest (modes 1 and 4): 0 compact every survivor into q64b; 1 or 2 a warp
// with at least compact_min survivors finishes them itself, with the six
// remaining bases (1) or the strong Lucas test (2), and compacts nothing.
template <int kImpl, int kMode, int kRest>
__global__ void __launch_bounds__(256) mr64_base2_kernel(const uint64_t* __restrict__ qn,
                                                         const uint32_t* __restrict__ qidx,
                                                         uint32_t* __restrict__ counters,
                                                         uint32_t* __restrict__ q64b,
                                                         uint8_t* __restrict__ out,
                                                         uint32_t compact_min, uint32_t mark) {
  extern __shared__ uint64_t s_tab[];  // mode 4 or kRest 1: 16 x blockDim
  const uint32_t count = *(volatile uint32_t*)&counters[0];
  const int lane = threadIdx.x & 31;
  // 32-survivor tasks: a warp's first task is fixed (global warp w takes
  // task w), later ones come from counters[3] (zeroed with the queues).  The
  // launch is one wave of resident blocks, and under a fixed stride the warps
  // the scheduler favours finish early while the rest run on with the SM
  // half empty (measured: 27 of 40 warps resident on average).  The next
  // task's atomic is issued before the current task runs, so its latency is
  // hidden, and warps without a first task issue none.
  const uint32_t first_tasks = gridDim.x * (blockDim.x >> 5) * 32u;
  uint32_t next = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u;
  while (next < count) {
    const uint32_t wbase = next;
    if (lane == 0) next = first_tasks + atomicAdd(&counters[3], 32u);
    const uint32_t i = wbase + lane;
    bool pass = false;
    uint64_t n = 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59 (prime) for lanes past the end
    if (i < count) {
      n = qn[i];
      if (kMode == 4) {
        const int nib = __reduce_max_sync(__activemask(), (unsigned)base2_nibbles(n));
        pass = base2_passes_win<kImpl>(n, s_tab + threadIdx.x, (int)blockDim.x, nib);
      } else if (kMode == 1) {
        const int nib = __reduce_max_sync(__activemask(), (unsigned)base2_nibbles(n));
        pass = base2_passes_shift<kImpl>(n, nib);
      } else {
        pass = base2_passes<kImpl>(n);
      }
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, pass);
    if (kRest != 0 && mask && (uint32_t)__popc(mask) >= compact_min) {
      // dense warp: finishing here costs fewer idle lanes than a queue round trip
      const uint64_t m = pass ? n : 0xFFFFFFFFFFFFFFC5ull;
      const bool prime = kRest == 2 ? lucas_warp<kImpl>(m, pass)
                                    : rest64_is_prime_warp<kImpl>(m, pass, s_tab + threadIdx.x,
                                                                  (int)blockDim.x);
      if (prime) out[qidx[i]] = 1;
    } else if (mask) {
      const int leader = __ffs(mask) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&counters[2], (uint32_t)__popc(mask));
      base = __shfl_sync(0xFFFFFFFFu, base, leader);
      if (pass) {
        q64b[base + __popc(mask & ((1u << lane) - 1u))] = i;
        if (mark) out[qidx[i]] = 1;  // prime unless a later base clears it (spread rest kernel)
      }
    }
    next = __shfl_sync(0xFFFFFFFFu, next, 0);
  }
}

// kLucas: the strong Lucas test (Baillie-PSW with the base-2 stage) instead
// of the six remaining Miller-Rabin bases.
template <int kImpl, bool kLucas, bool kSpread>
__global__ void __launch_bounds__(256) mr64_rest_kernel(const uint64_t* __restrict__ qn,
                                                        const uint32_t* __restrict__ qidx,
                                                        const uint32_t* __restrict__ q64b,
                                                        const uint32_t* __restrict__ counters,
                                                        uint8_t* __restrict__ out,
                                                        uint32_t spread_threads) {
  extern __shared__ uint64_t s_tab[];  // kTab x blockDim
  uint64_t* tab = s_tab + threadIdx.x;
  const int ld = blockDim.x;
  const uint32_t count = *(volatile const uint32_t*)&counters[2];
  // whole warps per iteration: both tests are warp-synchronous
  const int lane = threadIdx.x & 31;
  const uint32_t nthreads = gridDim.x * blockDim.x;
  const uint32_t first = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u;
  constexpr uint32_t kRestBases = kNumBases64 - 1;
  // kSpread: a queue shorter than the grid is spread over f = 6, 3 or 2
  // threads per survivor (6 / f bases each), so it takes the time of 6 / f
  // exponentiations instead of six; the base-2 kernel wrote 1 for every
  // survivor and a failing base writes 0.  Otherwise one survivor per thread,
  // and a survivor found prime gets its 1 here.
  if (kSpread && !kLucas) {
    // f from the threads the chunk could use (spread_threads, six per element
    // of the chunk up to the grid cap); the launch itself is capped at the
    // blocks that can be resident and strides over the pairs
    uint32_t f = 1;
    if ((uint64_t)count * kRestBases <= spread_threads) f = kRestBases;
    else if ((uint64_t)count * 3 <= spread_threads) f = 3;
    else if ((uint64_t)count * 2 <= spread_threads) f = 2;
    if (f > 1) {
      const int per = (int)(kRestBases / f);
      const uint32_t pairs = count * f;
      for (uint32_t wbase = first; wbase < pairs; wbase += nthreads) {
        const uint32_t g = wbase + lane;
        const bool valid = g < pairs;
        const uint32_t e = valid ? g / f : 0u;
        const uint32_t j = valid ? q64b[e] : 0u;
        const uint64_t n = valid ? qn[j] : 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59 for idle lanes
        const bool pass = bases_pass_warp<kImpl>(n, 1 + (int)(g - e * f) * per, per, tab, ld);
        if (valid && !pass) out[qidx[j]] = 0;
      }
      return;
    }
  }
  for (uint32_t wbase = first; wbase < count; wbase += nthreads) {
    const uint32_t i = wbase + lane;
    const bool valid = i < count;
    const uint32_t j = valid ? q64b[i] : 0u;
    const uint64_t n = valid ? qn[j] : 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59 for idle lanes
    const bool prime = kLucas ? lucas_warp<kImpl>(n, valid) : rest64_is_prime_warp<kImpl>(n, valid, tab, ld);
    if (kSpread) {
      if (valid && !prime) out[qidx[j]] = 0;
    } else if (prime) {
      out[qidx[j]] = 1;
    }
  }
}

__global__ void __launch_bounds__(256) mr32_kernel(const uint32_t* __restrict__ qn,
                                                   const uint32_t* __restrict__ qidx,
                                                   const uint32_t* __restrict__ counters,
                                                   uint8_t* __restrict__ out) {
  const uint32_t count = *(volatile const uint32_t*)&counters[1];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    if (mr32_is_prime(qn[i])) out[qidx[i]] = 1;
}

// Grid of a grid-stride kernel: at most the blocks that can be resident.
static unsigned resident_grid(const void* fn, unsigned block, size_t smem, int sm_count,
                              unsigned want) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)block, smem) != cudaSuccess ||
      per_sm < 1)
    return want;
  const unsigned cap = (unsigned)(sm_count * per_sm);
  return want < cap ? want : cap;
}

// Modes 1 and 4 run one wave of resident blocks (the kernel balances the
// warps itself); the table of mode 4 and the finishing of kRest 1 take
// 16 x block words of shared memory.
template <int kImpl, int kMode, int kRest>
static void launch_base2_win(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                             uint32_t compact_min, uint32_t mark, int sm_count, cudaStream_t s) {
  const size_t smem = (kMode == 4 || kRest == 1) ? (size_t)16 * block * sizeof(uint64_t) : 0;
  const void* fn = reinterpret_cast<const void*>(&mr64_base2_kernel<kImpl, kMode, kRest>);
  grid = resident_grid(fn, block, smem, sm_count, grid);
  mr64_base2_kernel<kImpl, kMode, kRest><<<grid, block, smem, s>>>(q.q64_n, q.q64_idx, q.counters,
                                                                   q.q64b, out, compact_min, mark);
}

template <int kImpl, int kMode>
static void launch_base2_mode(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                              int lucas, uint32_t compact_min, uint32_t mark, int sm_count,
                              cudaStream_t s) {
  if (compact_min > 32)
    launch_base2_win<kImpl, kMode, 0>(q, out, grid, block, compact_min, mark, sm_count, s);
  else if (lucas == 1)
    launch_base2_win<kImpl, kMode, 2>(q, out, grid, block, compact_min, mark, sm_count, s);
  else
    launch_base2_win<kImpl, kMode, 1>(q, out, grid, block, compact_min, mark, sm_count, s);
}

template <int kImpl>
static void launch_base2(const Queues& q, uint8_t* out, unsigned grid, unsigned block, int window,
                         int lucas, uint32_t compact_min, uint32_t mark, int sm_count,
                         cudaStream_t s) {
  if (window == 4) {
    launch_base2_mode<kImpl, 4>(q, out, grid, block, lucas, compact_min, mark, sm_count, s);
  } else if (window == 1) {
    launch_base2_mode<kImpl, 1>(q, out, grid, block, lucas, compact_min, mark, sm_count, s);
  } else {
    mr64_base2_kernel<kImpl, 0, 0><<<grid, block, 0, s>>>(q.q64_n, q.q64_idx, q.counters,
                                                          q.q64b, out, 33u, mark);
  }
}

// spread_grid > 0: launch the variant that spreads (survivor, base) pairs
// over the threads whenever the queue is at most a sixth of its threads.
template <int kImpl>
static void launch_rest(const Queues& q, uint8_t* out, unsigned grid, unsigned block, int lucas,
                        unsigned spread_grid, int sm_count, cudaStream_t s) {
  const size_t smem = (size_t)kTab * block * sizeof(uint64_t);
  if (lucas) {
    mr64_rest_kernel<kImpl, true, false><<<grid, block, 0, s>>>(q.q64_n, q.q64_idx, q.q64b, q.counters,
                                                                out, 0u);
  } else if (spread_grid) {
    // at most the blocks that can be resident: more would only queue up (and
    // cost their launch when the queue is empty)
    const uint32_t spread_threads = spread_grid * block;
    const void* fn = reinterpret_cast<const void*>(&mr64_rest_kernel<kImpl, false, true>);
    const unsigned g = resident_grid(fn, block, smem, sm_count, spread_grid);
    mr64_rest_kernel<kImpl, false, true><<<g, block, smem, s>>>(q.q64_n, q.q64_idx, q.q64b, q.counters,
                                                                out, spread_threads);
  } else {
    mr64_rest_kernel<kImpl, false, false><<<grid, block, smem, s>>>(q.q64_n, q.q64_idx, q.q64b,
                                                                   q.counters, out, 0u);
  }
}

// impl_b2 selects the arithmetic of the base-2 kernel, impl that of the
// six-base kernel (see MontOps).
static int launch_mr64(const Queues& q, uint8_t* out, unsigned grid, unsigned block, int impl,
                       int impl_b2, int window, int lucas, uint32_t compact_min, int sm_count,
                       unsigned spread_grid, cudaStream_t s, isprime_ctx* ctx) {
  int st = ISPRIME_OK;
  TimedLaunch tl;
  if (ctx && (st = launch_begin(ctx, ISPRIME_K_MR64_BASE2, s, &tl))) return st;
  const uint32_t cm = compact_min;
  // the spread rest kernel clears survivors that a later base rejects, so the
  // base-2 kernel marks its survivors prime first
  const uint32_t mark = (spread_grid != 0 && lucas != 1) ? 1u : 0u;
  if (lucas == 1) spread_grid = 0;
  switch (impl_b2) {
    case 1: launch_base2<1>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    case 2: launch_base2<2>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    case 3: launch_base2<3>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    case 4: launch_base2<4>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    case 5: launch_base2<5>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    case 6: launch_base2<6>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    case 7: launch_base2<7>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    case 8: launch_base2<8>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
    default: launch_base2<0>(q, out, grid, block, window, lucas, cm, mark, sm_count, s); break;
  }
  if (ctx && (st = launch_end(ctx, s, &tl, "mr64_base2_kernel"))) return st;
  if (ctx && (st = launch_begin(ctx, ISPRIME_K_MR64_REST, s, &tl))) return st;
  switch (impl) {
    case 1: launch_rest<1>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    case 2: launch_rest<2>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    case 3: launch_rest<3>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    case 4: launch_rest<4>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    case 5: launch_rest<5>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    case 6: launch_rest<6>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    case 7: launch_rest<7>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    case 8: launch_rest<8>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
    default: launch_rest<0>(q, out, grid, block, lucas, spread_grid, sm_count, s); break;
  }
  if (ctx) st = launch_end(ctx, s, &tl, "mr64_rest_kernel");
  return st;
}

int launch_mr(isprime_ctx* ctx, const Queues& q, uint8_t* out, uint64_t len, cudaStream_t s) {
  const uint32_t block = ctx->tune.mr_block;
  // The queues hold at most `len` elements (one per thread and pass), so a
  // short chunk gets a short grid.
  const uint64_t cap = (uint64_t)ctx->sm_count * ctx->tune.blocks_per_sm;
  const uint64_t want = (len + block - 1) / block;
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  // Chunks up to 2^22 elements take the rest kernel that can spread a short
  // queue over (survivor, base) pairs (it decides on the device from the
  // queue length); longer chunks take the variant without that mode, whose
  // register allocation suits long queues.
  const uint64_t want6 = (6 * len + block - 1) / block;  // six threads per element of the chunk
  const unsigned spread_grid =
      len <= ((uint64_t)1 << 22) ? (unsigned)(want6 < cap ? (want6 ? want6 : 1) : cap) : 0u;
  TimedLaunch tl;
  int st;
  if (sieve_cut(ctx) < (1ull << 32)) {
    if ((st = launch_begin(ctx, ISPRIME_K_MR32, s, &tl))) return st;
    mr32_kernel<<<grid, block, 0, s>>>(q.q32_n, q.q32_idx, q.counters, out);
    if ((st = launch_end(ctx, s, &tl, "mr32_kernel"))) return st;
  }
  return launch_mr64(q, out, grid, block, (int)ctx->tune.mont_impl,
                     (int)ctx->tune.mont_impl_base2, (int)ctx->tune.base2_window,
                     (int)ctx->tune.rest_test, ctx->tune.compact_min, ctx->sm_count, spread_grid,
                     s, ctx);
}

// Launch without a context (explicit grid and block and queue pointers);
// used by the allocation-free entry point.
int launch_mr_raw(const Queues& q, uint8_t* out, bool with_mr32, unsigned grid, unsigned block,
                  cudaStream_t s) {
  if (with_mr32) mr32_kernel<<<grid, block, 0, s>>>(q.q32_n, q.q32_idx, q.counters, out);
  // Montgomery formulation 6; base 2 by the binary schedule (its launch needs
  // no occupancy query, so no SM count)
  launch_mr64(q, out, grid, block, 6, 6, /*window=*/0, /*lucas=*/0, /*compact_min=*/33,
              /*sm_count=*/0, /*spread_grid=*/0, s, nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ISPRIME_OK : cuda_fail(e, "Miller-Rabin kernels");
}

}  // namespace ip
