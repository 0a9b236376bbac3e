// mr.cu -- deterministic Miller-Rabin on the compacted survivor queues.
//
// Sec. 2.1: n - 1 = 2^s d with d odd; n passes base a when a^d = 1 or
// a^(2^r d) = n - 1 for some r < s (the textbook strong condition; the
// printed "+-1" of Eq. 1 is read this way).  The seven bases of Eq. 4 decide
// every n < 2^64; {2, 7, 61} decide every n < 4,759,123,141.
//
// Kernels (each a grid-stride loop over a queue whose length is read on the
// device, so no host synchronisation separates the stages):
//   mr64_base2_kernel  a second trial stage (td2_groups: the primes after 53,
//                      on the queue's values, survivors staged per warp so
//                      the exponentiations run on full warps), then base 2 by
//                      4-bit windows where "multiply by 2^w" is x 2^w - q n
//                      with an estimated quotient (base2_window 1 or 2), or a
//                      Montgomery product with the table 2^w R (4), or binary
//                      with a modular doubling per set bit (0).  Passing
//                      elements (the primes and rare strong pseudoprimes) are
//                      compacted with warp ballots into a second queue, so the
//                      next kernel runs on dense warps of likely primes instead
//                      of idling behind early-exiting composites.  With the
//                      compaction threshold compact_min <= 32, a warp left with
//                      at least that many survivors finishes them itself.
//   mr64_rest_kernel   the six remaining bases, fixed-window exponentiation
//                      (3- or 4-bit, rest_window) with the per-thread window
//                      tables in shared memory, the bases one at a time or in
//                      pairs (rest_ilp).  On chunks of at most 2^22 elements a
//                      queue shorter than the grid is spread over 6, 3 or 2
//                      threads per survivor (the base-2 kernel then marks its
//                      survivors prime and a failing base clears the byte);
//                      otherwise one survivor per thread, writing 1 for primes.
//   mr32_kernel        bases 2, 7, 61 in 32-bit Montgomery arithmetic for
//                      survivors between the sieve cutover and 2^32.
// All arithmetic is in arith.cuh (ModExp / ModMultiply / ModAdd of
// Sec. 2.2-2.4 as Montgomery multiplication and doubling).
#include <string.h>

#include "device_common.cuh"
#include "internal.h"

namespace ip {

// Programmatic dependent launch (tuning pdl): the Miller-Rabin kernels may be
// launched while the previous kernel on the stream is still running; each
// waits here, before its first read of the queues, until that kernel has
// finished and its writes are visible.  Without the launch attribute the
// wait returns at once.
__device__ __forceinline__ void wait_for_producer() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static void launch_k(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                     cudaStream_t s, bool pdl, Args... args) {
  if (!pdl) {
    kernel<<<grid, block, smem, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// kMode: the base-2 schedule (the tuning field base2_window): 0 binary with
// a modular doubling per set bit, 1 4-bit windows with x 2^w mod n by a
// quotient estimated in single precision, 2 the same with the quotient
// estimated in integers, 4 4-bit windows with the table 2^w R in shared memory.
// kRest (modes 1 and 4): 0 compact every survivor into q64b; 1 or 2 a warp
// with at least compact_min survivors finishes them itself, with the six
// remaining bases (1) or the strong Lucas test (2), and compacts nothing.
// kIlp (mode 1, kRest 0): survivors per thread, 1 or 2 (two independent
// exponentiations per thread, base2_passes_shift_x2).
//
// The queue q64 has two regions (see classify.cu): [0, counters[0]) from the
// front and [cap - counters[1], cap) from the back.  When classify splits by
// s (n - 1 = 2^s d), the front holds s = 1 and the back s >= 2, so the
// strong-test tail, which a warp runs for its largest s, is empty for the
// front's warps.  Tasks of 32 * kIlp positions walk the front region (its
// last task padded) and then the back region.
//
// kTd2 > 0 (mode 1, kRest 0, kIlp 1): the second trial-division stage by the
// first kTd2 groups of c_td2 runs on every fetched task first, and the warp
// stages the values that survive it in its slice of shared memory (a stack of
// at most 63 positions and values); whenever 32 are staged, the warp runs the
// base-2 test on the top 32, so the exponentiations run on full warps while
// about a quarter of the queue never reaches them.  When no task is left, the
// warps of a block pool what their stacks still hold and run it as full
// batches.
template <int kImpl, int kMode, int kRest, int kIlp = 1, int kTd2 = 0>
__global__ void __launch_bounds__(256) mr64_base2_kernel(const uint64_t* __restrict__ qn,
                                                         const uint32_t* __restrict__ qidx,
                                                         uint32_t* __restrict__ counters,
                                                         uint32_t* __restrict__ q64b,
                                                         uint8_t* __restrict__ out,
                                                         uint32_t compact_min, uint32_t mark,
                                                         uint32_t cap) {
  extern __shared__ uint64_t s_tab[];  // mode 4 or kRest 1: 16 x blockDim
  constexpr uint32_t kTask = kTd2 > 0 ? 32u : 32u * kIlp;  // queue positions per task
  wait_for_producer();
  const uint32_t count_f = *(volatile uint32_t*)&counters[0];
  const uint32_t count_b = *(volatile uint32_t*)&counters[1];
  const uint32_t front_pad = (count_f + kTask - 1) / kTask * kTask;
  const uint32_t vcount = front_pad + count_b;  // virtual positions: front (padded), back
  const uint32_t back0 = cap - count_b;
  const int lane = threadIdx.x & 31;
  // Tasks: a warp's first task is fixed (global warp w takes task w), later
  // ones come from counters[3] (zeroed with the queues).  The launch is one
  // wave of resident blocks, and under a fixed stride the warps the scheduler
  // favours finish early while the rest run on with the SM half empty
  // (measured: 27 of 40 warps resident on average).  The next task's atomic
  // is issued before the current task runs, so its latency is hidden, and
  // warps without a first task issue none.
  const uint32_t first_tasks = gridDim.x * (blockDim.x >> 5) * kTask;
  uint32_t next = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kTask;
  // Appends the lanes with pass set to q64b (one atomic per warp) and, for the
  // spreading six-base kernel, marks them prime.
  auto append_passing = [&](bool pass, uint32_t pos) {
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, pass);
    if (!mask) return;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&counters[2], (uint32_t)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (pass) {
      const uint32_t k = base + __popc(mask & ((1u << lane) - 1u));
      if (IP_CHECK(k < cap, kChkQ64b)) q64b[k] = pos;
      if (mark && IP_CHECK(qidx[pos] < cap, kChkMrOut)) out[qidx[pos]] = 1;
    }
  };
  if constexpr (kTd2 > 0) {
    static_assert((kMode == 1 || kMode == 2) && kRest == 0 && (kIlp == 1 || kMode == 1),
                  "second trial stage: shift windows only (two per thread: the float estimate)");
    // A batch is kB = 32 kIlp values (kIlp per lane).  This warp's stack holds
    // fewer than kB plus one task: kStack values, then kStack positions; after
    // the block's stacks, the block's leftovers (fewer than kB per warp).
    constexpr int kB = 32 * kIlp, kStack = kB + 32;
    const int nwarps = (int)(blockDim.x >> 5), warp = (int)(threadIdx.x >> 5);
    uint64_t* st_n = s_tab + warp * (kStack + kStack / 2);
    uint32_t* st_pos = reinterpret_cast<uint32_t*>(st_n + kStack);
    uint64_t* left_n = s_tab + nwarps * (kStack + kStack / 2);
    uint32_t* left_pos = reinterpret_cast<uint32_t*>(left_n + kB * nwarps);
    __shared__ uint32_t s_left;
    if (threadIdx.x == 0) s_left = 0;
    __syncthreads();
    // base 2 on kB values of stack slots s0 + lane + 32 u (u < kIlp); lanes
    // past `cnt` values sit out (one value per lane) or test a prime and
    // report nothing (two per lane)
    auto run_batch = [&](const uint64_t* sn, const uint32_t* sp, int s0, int cnt) {
      uint64_t n[kIlp];
      uint32_t pos[kIlp];
      bool ok[kIlp];
#pragma unroll
      for (int u = 0; u < kIlp; ++u) {
        const int k = s0 + lane + 32 * u;
        ok[u] = lane + 32 * u < cnt;
        n[u] = ok[u] ? sn[k] : 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59 (prime) when idle
        pos[u] = ok[u] ? sp[k] : 0u;
      }
      __syncwarp();  // read before the next task's values overwrite the slots
      bool pass[kIlp];
      if constexpr (kIlp == 2) {
        const int nib = (int)__reduce_max_sync(
            0xFFFFFFFFu, (unsigned)max(base2_nibbles(n[0]), base2_nibbles(n[1])));
        base2_passes_shift_x2<kImpl>(n[0], n[1], nib, &pass[0], &pass[1]);
      } else {  // lanes without a value sit out (a full batch has none)
        pass[0] = false;
        if (ok[0]) {
          const int nib = (int)__reduce_max_sync(__activemask(), (unsigned)base2_nibbles(n[0]));
          pass[0] = base2_passes_shift<kImpl, kMode == 2>(n[0], nib);
        }
      }
#pragma unroll
      for (int u = 0; u < kIlp; ++u) append_passing(ok[u] && pass[u], pos[u]);
    };
    int held = 0;  // staged values, the same in every lane
    for (;;) {
      const bool have = next < vcount;
      if (have) {
        const uint32_t vbase = next;
        if (lane == 0) next = first_tasks + atomicAdd(&counters[3], kTask);
        const uint32_t v = vbase + lane;
        uint32_t pos;
        bool valid;
        if (vbase < front_pad) {
          pos = v;
          valid = v < count_f;
        } else {
          pos = back0 + (v - front_pad);
          valid = v < vcount;
        }
        valid = valid && IP_CHECK(pos < cap, kChkQ64Read);
        const uint64_t n = valid ? qn[pos] : 0ull;
        const bool keep = valid && !td2_divisible<kTd2>(n, c_td2);
        const unsigned km = __ballot_sync(0xFFFFFFFFu, keep);
        if (keep) {
          const int k = held + __popc(km & ((1u << lane) - 1u));
          if (IP_CHECK(k < kStack, kChkSmemQueue)) {
            st_n[k] = n;
            st_pos[k] = pos;
          }
        }
        held += __popc(km);
        next = __shfl_sync(0xFFFFFFFFu, next, 0);
        __syncwarp();
      }
      // full batches from the top of the stack
      while (held >= kB) {
        held -= kB;
        run_batch(st_n, st_pos, held, kB);
      }
      if (!have) break;
    }
    // No task left: the warps of the block pool what their stacks still hold
    // (fewer than kB each) and run it as full batches, about half as many
    // warp-batches as each warp running its own partial one.
    uint32_t at = 0;
    if (lane == 0 && held > 0) at = atomicAdd(&s_left, (uint32_t)held);
    at = __shfl_sync(0xFFFFFFFFu, at, 0);
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const int k = lane + 32 * u;
      if (k < held && IP_CHECK(at + k < (uint32_t)(kB * nwarps), kChkSmemQueue)) {
        left_n[at + k] = st_n[k];
        left_pos[at + k] = st_pos[k];
      }
    }
    __syncthreads();
    const uint32_t left = s_left;
    for (uint32_t b = (uint32_t)(kB * warp); b < left; b += (uint32_t)(kB * nwarps))
      run_batch(left_n, left_pos, (int)b, (int)min(left - b, (uint32_t)kB));
    return;
  }
  while (next < vcount) {
    const uint32_t vbase = next;
    if (lane == 0) next = first_tasks + atomicAdd(&counters[3], kTask);
    // queue positions of this lane's values (kIlp of them), valid or not
    uint32_t pos[kIlp];
    bool valid[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const uint32_t v = vbase + 32u * u + lane;
      if (vbase < front_pad) {
        pos[u] = v;
        valid[u] = v < count_f;
      } else {
        pos[u] = back0 + (v - front_pad);
        valid[u] = v < vcount;
      }
    }
    bool pass[kIlp];
    uint64_t n[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      pass[u] = false;
      valid[u] = valid[u] && IP_CHECK(pos[u] < cap, kChkQ64Read);
      n[u] = valid[u] ? qn[pos[u]] : 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59 (prime) when idle
    }
    if (kIlp == 2) {
      const int nib = (int)__reduce_max_sync(
          0xFFFFFFFFu, (unsigned)max(base2_nibbles(n[0]), base2_nibbles(n[kIlp - 1])));
      bool p0, p1;
      base2_passes_shift_x2<kImpl>(n[0], n[kIlp - 1], nib, &p0, &p1);
      pass[0] = valid[0] && p0;
      pass[kIlp - 1] = valid[kIlp - 1] && p1;
    } else if (valid[0]) {
      if (kMode == 4) {
        const int nib = __reduce_max_sync(__activemask(), (unsigned)base2_nibbles(n[0]));
        pass[0] = base2_passes_win<kImpl>(n[0], s_tab + threadIdx.x, (int)blockDim.x, nib);
      } else if (kMode == 1 || kMode == 2) {
        const int nib = __reduce_max_sync(__activemask(), (unsigned)base2_nibbles(n[0]));
        pass[0] = base2_passes_shift<kImpl, kMode == 2>(n[0], nib);
      } else {
        pass[0] = base2_passes<kImpl>(n[0]);
      }
    }
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const unsigned mask = __ballot_sync(0xFFFFFFFFu, pass[u]);
      if (kRest != 0 && mask && (uint32_t)__popc(mask) >= compact_min) {
        // dense warp: finishing here costs fewer idle lanes than a queue round trip
        const uint64_t m = pass[u] ? n[u] : 0xFFFFFFFFFFFFFFC5ull;
        const bool prime = kRest == 2 ? lucas_warp<kImpl>(m, pass[u])
                                      : rest64_is_prime_warp<kImpl>(m, pass[u], s_tab + threadIdx.x,
                                                                    (int)blockDim.x);
        if (prime && IP_CHECK(qidx[pos[u]] < cap, kChkMrOut)) out[qidx[pos[u]]] = 1;
      } else {
        // prime unless a later base clears it (spread rest kernel)
        append_passing(pass[u], pos[u]);
      }
    }
    next = __shfl_sync(0xFFFFFFFFu, next, 0);
  }
}

// kLucas: the strong Lucas test (Baillie-PSW with the base-2 stage) instead
// of the six remaining Miller-Rabin bases.  kW: window bits of the six
// exponentiations (3 or 4; the shared table holds 2^kW values per thread).
// kPair: one survivor per thread (kSpread: when the queue is too long to
// spread) takes the bases in pairs, two exponentiations interleaved per
// thread (rest64_is_prime_warp2), the second table after the first (2^kW
// more words per thread).
template <int kImpl, bool kLucas, bool kSpread, int kW = kWin, bool kPair = false>
__global__ void __launch_bounds__(256) mr64_rest_kernel(const uint64_t* __restrict__ qn,
                                                        const uint32_t* __restrict__ qidx,
                                                        const uint32_t* __restrict__ q64b,
                                                        const uint32_t* __restrict__ counters,
                                                        uint8_t* __restrict__ out,
                                                        uint32_t spread_threads, uint32_t cap) {
  extern __shared__ uint64_t s_tab[];  // 2^kW x blockDim
  uint64_t* tab = s_tab + threadIdx.x;
  const int ld = blockDim.x;
  wait_for_producer();
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
        uint32_t j = valid ? q64b[e] : 0u;
        if (!IP_CHECK(j < cap, kChkRestRead)) j = 0;
        const uint64_t n = valid ? qn[j] : 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59 for idle lanes
        const bool pass = bases_pass_warp<kImpl, kW>(n, 1 + (int)(g - e * f) * per, per, tab, ld);
        if (valid && !pass && IP_CHECK(qidx[j] < cap, kChkRestOut)) out[qidx[j]] = 0;
      }
      return;
    }
  }
  for (uint32_t wbase = first; wbase < count; wbase += nthreads) {
    const uint32_t i = wbase + lane;
    const bool valid = i < count;
    uint32_t j = valid ? q64b[i] : 0u;
    if (!IP_CHECK(j < cap, kChkRestRead)) j = 0;
    const uint64_t n = valid ? qn[j] : 0xFFFFFFFFFFFFFFC5ull;  // 2^64 - 59 for idle lanes
    bool prime;
    if constexpr (kLucas)
      prime = lucas_warp<kImpl>(n, valid);
    else if constexpr (kPair)
      prime = rest64_is_prime_warp2<kImpl, kW>(n, valid, tab, tab + (ld << kW), ld);
    else
      prime = rest64_is_prime_warp<kImpl, kW>(n, valid, tab, ld);
    if (!IP_CHECK(!valid || qidx[j] < cap, kChkRestOut)) {
    } else if (kSpread) {
      if (valid && !prime) out[qidx[j]] = 0;
    } else if (prime) {
      out[qidx[j]] = 1;
    }
  }
}

__global__ void __launch_bounds__(256) mr32_kernel(const uint32_t* __restrict__ qn,
                                                   const uint32_t* __restrict__ qidx,
                                                   const uint32_t* __restrict__ counters,
                                                   uint8_t* __restrict__ out, uint32_t cap) {
  wait_for_producer();
  const uint32_t count = *(volatile const uint32_t*)&counters[4];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    if (IP_CHECK(i < cap && qidx[i] < cap, kChkMr32) && mr32_is_prime(qn[i])) out[qidx[i]] = 1;
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

// How the Miller-Rabin stages of one chunk run (from the context's tuning).
struct MrOpts {
  int impl = 6;       // Montgomery formulation of the six-base kernel
  int impl_b2 = 6;    // and of the base-2 kernel
  int window = 1;     // base-2 schedule (base2_window)
  int lucas = 0;      // rest_test
  uint32_t compact_min = 33;
  int ilp = 1;        // base2_ilp
  int rest_win = 4;   // rest_window
  int b2_per_sm = 0;  // base2_blocks_per_sm (0: as many as fit)
  bool pdl = false;   // launch with programmatic stream serialization
  int td2 = 0;        // td2_groups: second trial stage in the base-2 kernel
  int rest_ilp = 1;   // six-base kernel: bases one at a time (1) or in pairs (2)
};

// Modes 1 and 4 run one wave of resident blocks (the kernel balances the
// warps itself); the table of mode 4 and the finishing of kRest 1 take
// 16 x block words of shared memory.
template <int kImpl, int kMode, int kRest, int kIlp, int kTd2 = 0>
static void launch_base2_win(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                             uint32_t compact_min, uint32_t mark, int sm_count, cudaStream_t s,
                             int per_sm_cap, bool pdl) {
  // the table of mode 4 and the finishing of kRest 1: 16 words per thread;
  // the second trial stage, per warp: a stack of 32 (kIlp + 1) values and
  // positions and 32 kIlp leftover slots, 1.5 words each
  const size_t smem = kTd2 > 0 ? (size_t)(48 * (kIlp + 1) + 48 * kIlp) * (block / 32) * sizeof(uint64_t)
                      : (kMode == 4 || kRest == 1) ? (size_t)16 * block * sizeof(uint64_t)
                                                   : 0;
  auto kern = mr64_base2_kernel<kImpl, kMode, kRest, kIlp, kTd2>;
  grid = resident_grid(reinterpret_cast<const void*>(kern), block, smem, sm_count, grid);
  if (per_sm_cap > 0 && sm_count > 0 && grid > (unsigned)(sm_count * per_sm_cap))
    grid = (unsigned)(sm_count * per_sm_cap);
  launch_k(kern, grid, block, smem, s, pdl, q.q64_n, q.q64_idx, q.counters, q.q64b, out,
           compact_min, mark, (uint32_t)q.capacity);
}

template <int kImpl, int kMode>
static void launch_base2_mode(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                              const MrOpts& o, uint32_t mark, int sm_count, cudaStream_t s) {
  if (o.compact_min > 32) {
    constexpr bool kFast = (kImpl == 6 || kImpl == 9 || kImpl == 16) && (kMode == 1 || kMode == 2);
    if constexpr (kFast) {
      // the second trial stage (formulations 6 and 9 and the counting build,
      // estimated-quotient windows, one survivor per thread)
      if constexpr (kMode == 1) {  // two staged values per lane (td2_groups 16 or 24)
        if (o.ilp == 2 && o.td2 == 16) {
          launch_base2_win<kImpl, 1, 0, 2, 16>(q, out, grid, block, o.compact_min, mark, sm_count, s,
                                               o.b2_per_sm, o.pdl);
          return;
        }
        if (o.ilp == 2 && o.td2 == 24) {
          launch_base2_win<kImpl, 1, 0, 2, 24>(q, out, grid, block, o.compact_min, mark, sm_count, s,
                                               o.b2_per_sm, o.pdl);
          return;
        }
      }
      if (o.td2 > 0) {
        switch (o.td2) {
          case 8: launch_base2_win<kImpl, kMode, 0, 1, 8>(q, out, grid, block, o.compact_min, mark,
                                                      sm_count, s, o.b2_per_sm, o.pdl); return;
          case 12: launch_base2_win<kImpl, kMode, 0, 1, 12>(q, out, grid, block, o.compact_min, mark,
                                                        sm_count, s, o.b2_per_sm, o.pdl); return;
          case 16: launch_base2_win<kImpl, kMode, 0, 1, 16>(q, out, grid, block, o.compact_min, mark,
                                                        sm_count, s, o.b2_per_sm, o.pdl); return;
          default: launch_base2_win<kImpl, kMode, 0, 1, 24>(q, out, grid, block, o.compact_min, mark,
                                                        sm_count, s, o.b2_per_sm, o.pdl); return;
        }
      }
      // two survivors per thread (float quotient estimate only)
      if (o.ilp == 2 && kMode == 1) {
        launch_base2_win<kImpl, 1, 0, 2>(q, out, grid, block, o.compact_min, mark, sm_count, s,
                                         o.b2_per_sm, o.pdl);
        return;
      }
    }
    launch_base2_win<kImpl, kMode, 0, 1>(q, out, grid, block, o.compact_min, mark, sm_count, s,
                                         o.b2_per_sm, o.pdl);
  } else if (o.lucas == 1) {
    launch_base2_win<kImpl, kMode, 2, 1>(q, out, grid, block, o.compact_min, mark, sm_count, s,
                                         o.b2_per_sm, o.pdl);
  } else {
    launch_base2_win<kImpl, kMode, 1, 1>(q, out, grid, block, o.compact_min, mark, sm_count, s,
                                         o.b2_per_sm, o.pdl);
  }
}

template <int kImpl>
static void launch_base2(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                         const MrOpts& o, uint32_t mark, int sm_count, cudaStream_t s) {
  if (o.window == 4) {
    launch_base2_mode<kImpl, 4>(q, out, grid, block, o, mark, sm_count, s);
  } else if (o.window == 1) {
    launch_base2_mode<kImpl, 1>(q, out, grid, block, o, mark, sm_count, s);
  } else if (o.window == 2) {
    launch_base2_mode<kImpl, 2>(q, out, grid, block, o, mark, sm_count, s);
  } else {
    launch_k(mr64_base2_kernel<kImpl, 0, 0>, grid, block, 0, s, o.pdl, q.q64_n, q.q64_idx,
             q.counters, q.q64b, out, 33u, mark, (uint32_t)q.capacity);
  }
}

// spread_grid > 0: launch the variant that spreads (survivor, base) pairs
// over the threads whenever the queue is at most a sixth of its threads.
template <int kImpl, int kW>
static void launch_rest_w(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                          unsigned spread_grid, int sm_count, cudaStream_t s, bool pdl,
                          bool pair = false) {
  const size_t smem = ((size_t)1 << kW) * block * sizeof(uint64_t);
  if (spread_grid) {
    // at most the blocks that can be resident: more would only queue up (and
    // cost their launch when the queue is empty)
    const uint32_t spread_threads = spread_grid * block;
    if (pair) {  // a queue too long to spread takes the bases in pairs
      auto kern = mr64_rest_kernel<kImpl, false, true, kW, true>;
      const unsigned g =
          resident_grid(reinterpret_cast<const void*>(kern), block, 2 * smem, sm_count, spread_grid);
      launch_k(kern, g, block, 2 * smem, s, pdl, q.q64_n, q.q64_idx, q.q64b, q.counters, out,
               spread_threads, (uint32_t)q.capacity);
      return;
    }
    const void* fn = reinterpret_cast<const void*>(&mr64_rest_kernel<kImpl, false, true, kW>);
    const unsigned g = resident_grid(fn, block, smem, sm_count, spread_grid);
    launch_k(mr64_rest_kernel<kImpl, false, true, kW>, g, block, smem, s, pdl, q.q64_n, q.q64_idx,
             q.q64b, q.counters, out, spread_threads, (uint32_t)q.capacity);
  } else if (pair) {
    launch_k(mr64_rest_kernel<kImpl, false, false, kW, true>, grid, block, 2 * smem, s, pdl,
             q.q64_n, q.q64_idx, q.q64b, q.counters, out, 0u, (uint32_t)q.capacity);
  } else {
    launch_k(mr64_rest_kernel<kImpl, false, false, kW>, grid, block, smem, s, pdl, q.q64_n,
             q.q64_idx, q.q64b, q.counters, out, 0u, (uint32_t)q.capacity);
  }
}

template <int kImpl>
static void launch_rest(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                        const MrOpts& o, unsigned spread_grid, int sm_count, cudaStream_t s) {
  if (o.lucas) {
    launch_k(mr64_rest_kernel<kImpl, true, false>, grid, block, 0, s, o.pdl, q.q64_n, q.q64_idx,
             q.q64b, q.counters, out, 0u, (uint32_t)q.capacity);
  } else if ((kImpl == 6 || kImpl == 9 || kImpl == 17) && o.rest_win == 3) {
    launch_rest_w<kImpl, 3>(q, out, grid, block, spread_grid, sm_count, s, o.pdl, o.rest_ilp == 2);
  } else {
    launch_rest_w<kImpl, kWin>(q, out, grid, block, spread_grid, sm_count, s, o.pdl);
  }
}

// impl_b2 selects the arithmetic of the base-2 kernel, impl that of the
// six-base kernel (see MontOps).
static int launch_mr64(const Queues& q, uint8_t* out, unsigned grid, unsigned block,
                       const MrOpts& o, int sm_count, unsigned spread_grid, cudaStream_t s,
                       isprime_ctx* ctx) {
  int st = ISPRIME_OK;
  TimedLaunch tl;
  if (ctx && (st = launch_begin(ctx, ISPRIME_K_MR64_BASE2, s, &tl))) return st;
  // the spread rest kernel clears survivors that a later base rejects, so the
  // base-2 kernel marks its survivors prime first
  const uint32_t mark = (spread_grid != 0 && o.lucas != 1) ? 1u : 0u;
  if (o.lucas == 1) spread_grid = 0;
  switch (o.impl_b2) {
    case 1: launch_base2<1>(q, out, grid, block, o, mark, sm_count, s); break;
    case 2: launch_base2<2>(q, out, grid, block, o, mark, sm_count, s); break;
    case 3: launch_base2<3>(q, out, grid, block, o, mark, sm_count, s); break;
    case 4: launch_base2<4>(q, out, grid, block, o, mark, sm_count, s); break;
    case 5: launch_base2<5>(q, out, grid, block, o, mark, sm_count, s); break;
    case 6: launch_base2<6>(q, out, grid, block, o, mark, sm_count, s); break;
    case 7: launch_base2<7>(q, out, grid, block, o, mark, sm_count, s); break;
    case 8: launch_base2<8>(q, out, grid, block, o, mark, sm_count, s); break;
    case 9: launch_base2<9>(q, out, grid, block, o, mark, sm_count, s); break;
    case 16: launch_base2<16>(q, out, grid, block, o, mark, sm_count, s); break;
    default: launch_base2<0>(q, out, grid, block, o, mark, sm_count, s); break;
  }
  if (ctx && (st = launch_end(ctx, s, &tl, "mr64_base2_kernel"))) return st;
  // compact_min <= 1 with a windowed base-2 schedule: every warp finishes its
  // own passers, nothing is compacted, and the six-base kernel has no work
  if (o.compact_min <= 1 && o.window != 0) return st;
  if (ctx && (st = launch_begin(ctx, ISPRIME_K_MR64_REST, s, &tl))) return st;
  switch (o.impl) {
    case 1: launch_rest<1>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 2: launch_rest<2>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 3: launch_rest<3>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 4: launch_rest<4>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 5: launch_rest<5>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 6: launch_rest<6>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 7: launch_rest<7>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 8: launch_rest<8>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 9: launch_rest<9>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    case 17: launch_rest<17>(q, out, grid, block, o, spread_grid, sm_count, s); break;
    default: launch_rest<0>(q, out, grid, block, o, spread_grid, sm_count, s); break;
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
    launch_k(mr32_kernel, grid, block, 0, s, ctx->tune.pdl != 0 && !ctx->timing, q.q32_n, q.q32_idx,
             q.counters, out, (uint32_t)q.capacity);
    if ((st = launch_end(ctx, s, &tl, "mr32_kernel"))) return st;
  }
  MrOpts o;
  o.impl = (int)ctx->tune.mont_impl;
  o.impl_b2 = (int)ctx->tune.mont_impl_base2;
  o.window = (int)ctx->tune.base2_window;
  o.lucas = (int)ctx->tune.rest_test;
  o.compact_min = ctx->tune.compact_min;
  o.ilp = (int)ctx->tune.base2_ilp;
  o.rest_win = (int)ctx->tune.rest_window;
  o.b2_per_sm = (int)ctx->tune.base2_blocks_per_sm;
  o.pdl = ctx->tune.pdl != 0 && !ctx->timing;  // timing events between launches would serialise them
  o.td2 = (int)ctx->tune.td2_groups;
  o.rest_ilp = (int)ctx->tune.rest_ilp;
  // Short chunks: every warp of the base-2 kernel finishes its own passers
  // and the six-base kernel is not launched (one launch less per call, where
  // launches, not arithmetic, set the time).
  if (ctx->tune.inplace_max_log2 != 0 && len <= ((uint64_t)1 << ctx->tune.inplace_max_log2) &&
      o.window != 0)
    o.compact_min = 1;
  if (ctx->count_ops) {  // isprime_count_ops: formulation 6 with its operations counted
    o.impl_b2 = 16;
    o.impl = 17;
  }
  return launch_mr64(q, out, grid, block, o, ctx->sm_count, spread_grid, s, ctx);
}

// Launch without a context (explicit grid and block and queue pointers);
// used by the allocation-free entry point.
int launch_mr_raw(const Queues& q, uint8_t* out, bool with_mr32, unsigned grid, unsigned block,
                  cudaStream_t s) {
  if (with_mr32)
    mr32_kernel<<<grid, block, 0, s>>>(q.q32_n, q.q32_idx, q.counters, out, (uint32_t)q.capacity);
  // Montgomery formulation 6; base 2 by the binary schedule (its launch needs
  // no occupancy query, so no SM count)
  MrOpts o;
  o.window = 0;
  launch_mr64(q, out, grid, block, o, /*sm_count=*/0, /*spread_grid=*/0, s, nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ISPRIME_OK : cuda_fail(e, "Miller-Rabin kernels");
}

IP_CHECK_READER(check_read_mr)

// The operation counters of this translation unit (arith.cuh, g_ip_ops):
// out receives [stage][kind][warp issues, active lanes] summed over the
// spread copies; reset clears them.  Synchronous on the current device.
int op_counts_read(unsigned long long out[2][kOpKinds][2], bool reset) {
  unsigned long long h[2][kOpKinds][2][kOpSpread];
  IP_CUDA(cudaMemcpyFromSymbol(h, g_ip_ops, sizeof h));
  for (int st = 0; st < 2; ++st)
    for (int k = 0; k < kOpKinds; ++k)
      for (int j = 0; j < 2; ++j) {
        unsigned long long t = 0;
        for (int i = 0; i < kOpSpread; ++i) t += h[st][k][j][i];
        out[st][k][j] = t;
      }
  if (reset) {
    memset(h, 0, sizeof h);
    IP_CUDA(cudaMemcpyToSymbol(g_ip_ops, h, sizeof h));
  }
  return ISPRIME_OK;
}

}  // namespace ip
