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
// Loads are 16-byte vector loads (coalesced, eight elements per thread per
// tile); queue appends are warp-aggregated (one atomic per queue and warp).
#include "device_common.cuh"
#include "internal.h"

namespace ip {

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
  int d = ok ? classify_value<-1>(v, a) : kComposite;
  if (!ok && a.invalid) atomicAdd(a.invalid, 1ull);
  if (!ok && a.invalid_ctx) atomicAdd(a.invalid_ctx, 1ull);
  if (IP_CHECK(i < a.n, kChkOut)) a.out[i] = (uint8_t)(d == kPrime);
  if (d == kMR64) {
    // the front size is the low half of the 64-bit word counters[0..1]
    const uint32_t pos =
        (uint32_t)atomicAdd(reinterpret_cast<unsigned long long*>(a.counters), 1ull);
    if (IP_CHECK(pos < a.q64_cap, kChkQ64Front)) {
      a.q64_n[pos] = v;
      a.q64_idx[pos] = (uint32_t)i;
    }
  } else if (d == kMR32) {
    const uint32_t pos = atomicAdd(&a.counters[4], 1u);
    if (IP_CHECK(pos < a.q64_cap, kChkQ32)) {
      a.q32_n[pos] = (uint32_t)v;
      a.q32_idx[pos] = (uint32_t)i;
    }
  }
}

constexpr int kPairsPerThread = 4;  // 8 elements per thread per tile

// One tile = blockDim * kPairsPerThread pairs.  Pair p covers the elements
// head + 2p and head + 2p + 1.  Survivors of a tile are appended to the
// queues with one atomic per queue per warp.  40 registers give
// six 256-thread blocks per SM (measured: 0.115 ms per 2^24 large values,
// 0.547 ms per 2^26 mixed values, against 0.117 / 0.596 ms at 45).
// kFold: fold level of the 64-bit trial division (classify_value).
// kSplit: 64-bit survivors with n = 3 (mod 4) (s = 1 in n - 1 = 2^s d) are
// appended to q64 from the front, the others (s >= 2) from the back end
// (position q64_cap - 1 - k), so that the base-2 kernel's warps of the front
// region share s = 1 and skip the strong-test tail; without kSplit every
// survivor goes to the front.
template <typename T, int kNtd, int kFold = 0, bool kSplit = false>
__global__ void __maxnreg__(40) classify_kernel(ClassifyArgs a) {
  const uint64_t head = a.head;
  const uint64_t npairs = (a.n - head) / 2;
  const uint64_t tile_pairs = (uint64_t)blockDim.x * kPairsPerThread;
  const uint64_t ntiles = (npairs + tile_pairs - 1) / tile_pairs;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint64_t v[2 * kPairsPerThread];
    uint32_t dm = 0;     // the eight decisions, two bits each (element j at bits 2j, 2j+1)
    uint32_t sneed = 0;  // elements whose answer is a sieve bit (bit j), looked up below
    uint32_t nbad = 0;
    uint32_t s1 = 0;     // kSplit: n = 3 (mod 4) marks at the codes' even bit positions (2j)
#pragma unroll
    for (int k = 0; k < kPairsPerThread; ++k) {
      const uint64_t p = tile * tile_pairs + (uint64_t)k * blockDim.x + threadIdx.x;
      v[2 * k] = v[2 * k + 1] = 0;
      if (p < npairs) {
        bool ok0, ok1;
        Loader<T>::pair(a.in, head + 2 * p, &v[2 * k], &v[2 * k + 1], &ok0, &ok1);
        if (kSplit)
          s1 |= (((uint32_t)v[2 * k] >> 1) & 1u) << (4 * k) |
                (((uint32_t)v[2 * k + 1] >> 1) & 1u) << (4 * k + 2);
        const int d0 =
            ok0 ? classify_value<kNtd, ClassifyArgs, true, kFold>(v[2 * k], a) : kComposite;
        const int d1 =
            ok1 ? classify_value<kNtd, ClassifyArgs, true, kFold>(v[2 * k + 1], a) : kComposite;
        nbad += (uint32_t)!ok0 + (uint32_t)!ok1;
        sneed |= ((uint32_t)(d0 == kSieveLookup) << (2 * k)) |
                 ((uint32_t)(d1 == kSieveLookup) << (2 * k + 1));
        dm |= ((uint32_t)(d0 & 3) << (4 * k)) | ((uint32_t)(d1 & 3) << (4 * k + 2));
      }
    }
    // The sieve lookups of the tile's elements, all in flight together
    // (kSieveLookup & 3 == kComposite, so a set bit turns the code to kPrime).
    static_assert((kSieveLookup & 3) == kComposite, "deferred lookups start as composite");
    if (sneed) {
#pragma unroll
      for (int e = 0; e < 2 * kPairsPerThread; ++e)
        if ((sneed >> e) & 1u)
          dm |= ((__ldg(a.sieve + (v[e] >> 6)) >> ((uint32_t)(v[e] >> 1) & 31u)) & 1u) << (2 * e);
    }
#pragma unroll
    for (int k = 0; k < kPairsPerThread; ++k) {
      const uint64_t p = tile * tile_pairs + (uint64_t)k * blockDim.x + threadIdx.x;
      if (p < npairs) {
        const uint64_t i0 = head + 2 * p;
        const uint8_t o0 = (uint8_t)(((dm >> (4 * k)) & 3u) == kPrime);
        const uint8_t o1 = (uint8_t)(((dm >> (4 * k + 2)) & 3u) == kPrime);
        if (!IP_CHECK(i0 + 1 < a.n, kChkOut)) {
        } else if (a.pair_store) {
          *reinterpret_cast<uint16_t*>(a.out + i0) = (uint16_t)(o0 | (o1 << 8));
        } else {
          a.out[i0] = o0;
          a.out[i0 + 1] = o1;
        }
      }
    }
    // kMR64 = 0b10, kMR32 = 0b11: count the codes by their two bits
    static_assert(kComposite == 0 && kPrime == 1 && kMR64 == 2 && kMR32 == 3, "2-bit decision codes");
    const uint32_t dhi = (dm >> 1) & 0x5555u, dlo = dm & 0x5555u;
    const uint32_t m64 = dhi & ~dlo, n32 = __popc(dhi & dlo);
    const uint32_t n64f = __popc(kSplit ? (m64 & s1) : m64);
    const uint32_t n64b = kSplit ? __popc(m64 & ~s1) : 0u;
    // Warp-aggregated appends: the three counts (at most 8 per thread, 256 per
    // warp) packed in 10-bit fields, an exclusive scan over the warp, and one
    // atomic per queue per warp (no barrier, no shared memory).
    const int lane = threadIdx.x & 31;
    const uint32_t packed = n64f | (n64b << 10) | (n32 << 20);
    uint32_t incl = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t pre = incl - packed;
    const uint32_t wtot = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t bf = 0, bb = 0, b32 = 0;
    if (lane == 0) {
      const uint32_t tf = wtot & 0x3FFu, tb = (wtot >> 10) & 0x3FFu, t32 = wtot >> 20;
      // front and back sizes in one 64-bit word: one atomic for both regions
      if (tf | tb) {
        const unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(a.counters),
                                                 (unsigned long long)tf | ((unsigned long long)tb << 32));
        bf = (uint32_t)old;
        bb = (uint32_t)(old >> 32);
      }
      if (t32) b32 = atomicAdd(&a.counters[4], t32);
    }
    if (a.invalid || a.invalid_ctx) {
      const unsigned bad = __reduce_add_sync(0xFFFFFFFFu, nbad);
      if (lane == 0 && bad) {
        if (a.invalid) atomicAdd(a.invalid, (unsigned long long)bad);
        if (a.invalid_ctx) atomicAdd(a.invalid_ctx, (unsigned long long)bad);
      }
    }
    uint32_t pos64 = __shfl_sync(0xFFFFFFFFu, bf, 0) + (pre & 0x3FFu);
    uint32_t posb = __shfl_sync(0xFFFFFFFFu, bb, 0) + ((pre >> 10) & 0x3FFu);
    uint32_t pos32 = __shfl_sync(0xFFFFFFFFu, b32, 0) + (pre >> 20);
#pragma unroll
    for (int k = 0; k < kPairsPerThread; ++k) {
      const uint64_t p = tile * tile_pairs + (uint64_t)k * blockDim.x + threadIdx.x;
      const uint32_t i0 = (uint32_t)(head + 2 * p);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * k + h;
        const int dj = (int)((dm >> (2 * j)) & 3u);
        if (dj == kMR64) {
          // the front slot for s = 1 (or without the split), else the back one;
          // one store path either way, so the warp does not split here
          const bool front = !kSplit || ((s1 >> (2 * j)) & 1u);
          const uint32_t slot = front ? pos64 : a.q64_cap - 1u - posb;
          if (IP_CHECK(front ? pos64 < a.q64_cap : posb < a.q64_cap,
                       front ? kChkQ64Front : kChkQ64Back)) {
            a.q64_n[slot] = v[j];
            a.q64_idx[slot] = i0 + h;
          }
          pos64 += front ? 1u : 0u;
          posb += front ? 0u : 1u;
        } else if (dj == kMR32) {
          if (IP_CHECK(pos32 < a.q64_cap, kChkQ32)) {
            a.q32_n[pos32] = (uint32_t)v[j];
            a.q32_idx[pos32] = i0 + h;
          }
          ++pos32;
        }
      }
    }
  }
  // Alignment head (at most one element) and odd tail (at most one).
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (uint64_t i = 0; i < head; ++i) classify_single<T>(a, i);
    for (uint64_t i = head + 2 * npairs; i < a.n; ++i) classify_single<T>(a, i);
  }
}

// Trial-division counts with a compiled specialisation; other counts use
// the runtime-count kernel.
// The fold levels and the s-split are compiled for the default count (15,
// the odd primes 3..53, the primes fold_width knows); other counts take the
// unfolded, unsplit kernel (the results are the same either way).
template <typename T>
static void launch_classify_kernel(const ClassifyArgs& a, unsigned grid, unsigned block,
                                   cudaStream_t s) {
  if (a.ntd == 15 && (a.fold != 0 || a.split != 0)) {
    const int key = (int)a.fold * 2 + (a.split ? 1 : 0);
    switch (key) {
      case 1: classify_kernel<T, 15, 0, true><<<grid, block, 0, s>>>(a); return;
      case 2: classify_kernel<T, 15, 1, false><<<grid, block, 0, s>>>(a); return;
      case 3: classify_kernel<T, 15, 1, true><<<grid, block, 0, s>>>(a); return;
      case 4: classify_kernel<T, 15, 2, false><<<grid, block, 0, s>>>(a); return;
      case 5: classify_kernel<T, 15, 2, true><<<grid, block, 0, s>>>(a); return;
      case 6: classify_kernel<T, 15, 3, false><<<grid, block, 0, s>>>(a); return;
      default: classify_kernel<T, 15, 3, true><<<grid, block, 0, s>>>(a); return;
    }
  }
  switch (a.ntd) {
    case 0: classify_kernel<T, 0><<<grid, block, 0, s>>>(a); break;
    case 7: classify_kernel<T, 7><<<grid, block, 0, s>>>(a); break;
    case 11: classify_kernel<T, 11><<<grid, block, 0, s>>>(a); break;
    case 15: classify_kernel<T, 15><<<grid, block, 0, s>>>(a); break;
    case 23: classify_kernel<T, 23><<<grid, block, 0, s>>>(a); break;
    case 31: classify_kernel<T, 31><<<grid, block, 0, s>>>(a); break;
    default: classify_kernel<T, -1><<<grid, block, 0, s>>>(a); break;
  }
}

template <typename T>
static int launch_classify(isprime_ctx* ctx, const ClassifyArgs& a, cudaStream_t s, int kid,
                           const char* name) {
  const uint32_t block = ctx->tune.classify_block;
  const uint64_t npairs = (a.n - a.head) / 2;
  const uint64_t tile_pairs = (uint64_t)block * kPairsPerThread;
  uint64_t want = (npairs + tile_pairs - 1) / tile_pairs;
  const uint64_t cap = (uint64_t)ctx->sm_count * ctx->tune.blocks_per_sm;
  unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  TimedLaunch tl;
  int st = launch_begin(ctx, kid, s, &tl);
  if (st) return st;
  launch_classify_kernel<T>(a, grid, block, s);
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
  launch_classify_kernel<uint64_t>(a, grid, block, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ISPRIME_OK : cuda_fail(e, "classify_kernel<u64>");
}

IP_CHECK_READER(check_read_classify)

uint64_t td_square_for(uint32_t ntd) {
  const uint64_t next = ntd < (uint32_t)kMaxTdPrimes ? kTdPrimeList[ntd] : kTdNextPrimeAfterList;
  return next * next;
}

}  // namespace ip
