// range.cu -- primality of every integer in a window [lo, lo + count).
//
// The paper's array results are mostly incrementing sequences 1:N (Table 3)
// and a window of consecutive integers (Table 5, the Unix seconds of 2021);
// for them no input array is needed.  Two kernels:
//   range_expand_kernel  values below the resident sieve limit S: each output
//                        byte is one bit of the bitmap (Sec. 6.1.3's lookup),
//                        four bytes per thread, streaming.
//   range_sieve_kernel   values >= S: one block sieves a segment of the
//                        window in shared memory by every odd prime below
//                        2^16 (Sec. 1's sieve, applied to a window).  A value
//                        below 65537^2 that survives is prime; a survivor
//                        above it goes to the 64-bit Miller-Rabin queue, and
//                        the base-2 and six-base kernels of mr.cu finish it.
#include <algorithm>

#include "device_common.cuh"
#include "internal.h"

namespace ip {

// Segments: 512 words (32,768 integers) per block; windows too short to give
// every SM a few such blocks take 64-word segments (4,096 integers), which
// repeat the per-prime set-up eight times as often but fill the GPU.
constexpr int kRangeSegWords = 512;                 // 16,384 odd values per segment
constexpr int kRangeSegInts = kRangeSegWords * 64;  // integers covered by a segment
constexpr int kRangeSegWordsSmall = 64;
constexpr int kRangeThreads = 256;
constexpr uint64_t kSieveComplete = 65537ull * 65537ull;  // all primes < 2^16 sieve below this

struct RangeArgs {
  uint64_t lo;            // first value of this chunk
  uint64_t count;         // values in this chunk (lo + count <= 2^64)
  uint8_t* out;           // out[i] <-> lo + i
  const uint32_t* primes; // odd primes below 2^16, ascending
  const uint32_t* nprimes;
  uint64_t* q64_n;
  uint32_t* q64_idx;
  uint32_t* counters;
  const uint32_t* sieve;  // resident bitmap (expand kernel)
  uint32_t q64_cap;       // capacity of the survivor queue
};

// Single-thread expansion of a few values (alignment head and tail).
__global__ void range_expand_scalar_kernel(RangeArgs a) {
  for (uint64_t i = 0; i < a.count; ++i) {
    const uint64_t v = a.lo + i;
    a.out[i] = (v & 1) ? (uint8_t)((a.sieve[v >> 6] >> ((uint32_t)(v >> 1) & 31u)) & 1u)
                       : (uint8_t)(v == 2);
  }
}

// Spreads the 4 low bits of x into bytes 0, 2, 4, 6 of a 64-bit word (the
// shifted copies 1, 2^15, 2^30, 2^45 of x do not overlap, so no carries).
__device__ __forceinline__ uint64_t spread4(uint32_t x) {
  return ((uint64_t)(x & 15u) * 0x0000200040008001ull) & 0x0001000100010001ull;
}

// Sixteen values per thread: their eight odd values are eight consecutive
// bits of the bitmap, spread into the odd (or even) bytes of one 16-byte
// store.  a.count is a multiple of 16 and a.out is 16-byte aligned.
__global__ void __launch_bounds__(256) range_expand_kernel(RangeArgs a) {
  const uint64_t nv = a.count / 16;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v0 = a.lo + 16 * t;
    const uint64_t b0 = v0 >> 1;  // bit of the first odd value at or after v0
    const uint64_t w = b0 >> 5;
    // the next word only when the 8 bits cross into it (it then lies below S)
    const uint32_t next = ((b0 & 31) > 24) ? __ldg(a.sieve + w + 1) : 0u;
    const uint64_t pair = ((uint64_t)next << 32) | __ldg(a.sieve + w);
    const uint32_t bits = (uint32_t)(pair >> (b0 & 31)) & 0xFFu;
    uint64_t lo8 = spread4(bits), hi8 = spread4(bits >> 4);
    if (!(v0 & 1)) {  // odd values sit at the odd offsets 1, 3, ..., 15
      lo8 <<= 8;
      hi8 <<= 8;
    }
    if (v0 <= 2 && 2 < v0 + 16) lo8 |= 1ull << (8 * (2 - v0));  // the even prime
    uint4 q;
    q.x = (uint32_t)lo8;
    q.y = (uint32_t)(lo8 >> 32);
    q.z = (uint32_t)hi8;
    q.w = (uint32_t)(hi8 >> 32);
    *reinterpret_cast<uint4*>(a.out + 16 * t) = q;
  }
}

__device__ __forceinline__ void range_clear(uint32_t* seg, uint32_t j) {
  atomicAnd(&seg[j >> 5], ~(1u << (j & 31)));
}

// Block b sieves the integers [S0, S0 + kSegInts), S0 = even base of the
// chunk + b * kSegInts.  Bit j of the segment <-> the odd value S0 + 2j + 1.
template <int kSegWords>
__global__ void __launch_bounds__(kRangeThreads) range_sieve_kernel(RangeArgs a) {
  constexpr uint32_t kSegInts = kSegWords * 64;
  __shared__ uint32_t seg[kSegWords];
  __shared__ uint32_t s_scan[33];
  __shared__ uint32_t s_base;
  const uint32_t tid = threadIdx.x;
  const uint64_t base0 = a.lo & ~1ull;
  const uint64_t S0 = base0 + (uint64_t)blockIdx.x * kSegInts;
  // last value of the chunk and of this segment (no overflow: the window ends at or below 2^64 - 1)
  const uint64_t last = a.lo + (a.count - 1);
  const uint64_t seg_last = (last - S0 < (uint64_t)kSegInts) ? last : S0 + kSegInts - 1;

  for (uint32_t w = tid; w < kSegWords; w += kRangeThreads) seg[w] = 0xFFFFFFFFu;
  __syncthreads();
  // cross off odd multiples m >= max(p^2, S0) of every odd prime p with p^2 <= seg_last
  const uint32_t np = *a.nprimes;
  const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = kRangeThreads / 32;
  auto first_bit = [&](uint64_t p, uint32_t* j0) -> bool {
    // offset of the first multiple of p at or above S0 that is odd and >= p^2
    uint64_t off = (p - S0 % p) % p;
    if (!(off & 1)) off += p;  // S0 even, p odd: an even offset gives an even multiple
    const uint64_t p2 = p * p;
    if (S0 < p2 && S0 + off < p2) off = p2 - S0;  // p2 - S0 is odd here
    if (off >= (uint64_t)kSegInts) return false;
    *j0 = (uint32_t)((off - 1) >> 1);
    return true;
  };
  for (uint32_t i = warp; i < np; i += nwarps) {  // warp per prime: small primes, many multiples
    const uint64_t p = a.primes[i];
    if (p * p > seg_last) break;
    if (p >= 2048) break;
    uint32_t j0;
    if (!first_bit(p, &j0)) continue;
    for (uint32_t j = j0 + lane * (uint32_t)p; j < kSegWords * 32u; j += 32u * (uint32_t)p)
      range_clear(seg, j);
  }
  uint32_t i_split = 0;
  {
    uint32_t lo_i = 0, hi_i = np;
    while (lo_i < hi_i) {
      const uint32_t mid = (lo_i + hi_i) >> 1;
      if (a.primes[mid] < 2048) lo_i = mid + 1; else hi_i = mid;
    }
    i_split = lo_i;
  }
  for (uint32_t i = i_split + tid; i < np; i += kRangeThreads) {  // thread per prime
    const uint64_t p = a.primes[i];
    if (p * p > seg_last) break;
    uint32_t j0;
    if (!first_bit(p, &j0)) continue;
    for (uint32_t j = j0; j < kSegWords * 32u; j += (uint32_t)p) range_clear(seg, j);
  }
  __syncthreads();

  // Outputs: thread t writes values S0 + t, S0 + t + B, ... (coalesced bytes);
  // survivors that the sieve cannot decide are appended to the queue.
  for (uint32_t r = 0; r < (uint32_t)kSegInts; r += kRangeThreads) {
    const uint64_t off = r + tid;
    const uint64_t v = S0 + off;
    const bool inside = off <= seg_last - S0 && v >= a.lo;
    bool mr = false;
    if (inside) {
      uint8_t o;
      if (v < 2) o = 0;
      else if (!(v & 1)) o = (v == 2);
      else o = (uint8_t)((seg[(uint32_t)(off >> 1) >> 5] >> ((uint32_t)(off >> 1) & 31u)) & 1u);
      if (o && v >= kSieveComplete) {
        mr = true;
        o = 0;
      }
      if (IP_CHECK(v - a.lo < a.count, kChkRangeOut)) a.out[v - a.lo] = o;
    }
    // block-aggregated append of the undecided survivors
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, mr);
    if (lane == 0) s_scan[warp] = __popc(bal);
    __syncthreads();
    if (tid == 0) {
      uint32_t tot = 0;
      for (uint32_t w = 0; w < nwarps; ++w) {
        const uint32_t c = s_scan[w];
        s_scan[w] = tot;
        tot += c;
      }
      s_base = tot ? atomicAdd(&a.counters[0], tot) : 0u;
    }
    __syncthreads();
    if (mr) {
      const uint32_t pos = s_base + s_scan[warp] + __popc(bal & ((1u << lane) - 1u));
      if (IP_CHECK(pos < a.q64_cap, kChkRangeQueue)) {
        a.q64_n[pos] = v;
        a.q64_idx[pos] = (uint32_t)(v - a.lo);
      }
    }
    __syncthreads();
  }
}

// Expands [a.lo, a.lo + a.count) from the bitmap: an unaligned head and a
// short tail singly, the aligned body sixteen values per thread.
int launch_range_expand(isprime_ctx* ctx, const RangeArgs& a, cudaStream_t s) {
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_RANGE, s, &tl);
  if (st) return st;
  uint64_t head = (16 - ((uintptr_t)a.out & 15)) & 15;
  if (head > a.count) head = a.count;
  const uint64_t body = (a.count - head) & ~(uint64_t)15;
  const uint64_t tail = a.count - head - body;
  RangeArgs h = a;
  if (head) {
    h.count = head;
    range_expand_scalar_kernel<<<1, 1, 0, s>>>(h);
  }
  if (body) {
    RangeArgs b = a;
    b.lo = a.lo + head;
    b.out = a.out + head;
    b.count = body;
    const uint64_t want = (body / 16 + 255) / 256;
    const uint64_t cap = (uint64_t)ctx->sm_count * 16;
    range_expand_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(b);
  }
  if (tail) {
    RangeArgs t = a;
    t.lo = a.lo + head + body;
    t.out = a.out + head + body;
    t.count = tail;
    range_expand_scalar_kernel<<<1, 1, 0, s>>>(t);
  }
  return launch_end(ctx, s, &tl, "range_expand_kernel");
}

int launch_range_sieve(isprime_ctx* ctx, const RangeArgs& a, cudaStream_t s) {
  const uint64_t base0 = a.lo & ~1ull;
  const uint64_t last = a.lo + (a.count - 1);
  const uint64_t nseg = (last - base0) / kRangeSegInts + 1;
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_RANGE, s, &tl);
  if (st) return st;
  if (nseg < 4 * (uint64_t)ctx->sm_count) {
    constexpr uint64_t kSmallInts = (uint64_t)kRangeSegWordsSmall * 64;
    const uint64_t nsmall = (last - base0) / kSmallInts + 1;
    range_sieve_kernel<kRangeSegWordsSmall><<<(unsigned)nsmall, kRangeThreads, 0, s>>>(a);
  } else {
    range_sieve_kernel<kRangeSegWords><<<(unsigned)nseg, kRangeThreads, 0, s>>>(a);
  }
  return launch_end(ctx, s, &tl, "range_sieve_kernel");
}

IP_CHECK_READER(check_read_range)

int range_run(isprime_ctx* ctx, uint64_t lo, uint64_t count, uint8_t* d_out, cudaStream_t s) {
  uint64_t done = 0;
  int st = ISPRIME_OK;
  // Part below the resident sieve limit: bitmap expansion.
  if (lo < ctx->sieve_limit) {
    const uint64_t n1 = (ctx->sieve_limit - lo < count) ? ctx->sieve_limit - lo : count;
    RangeArgs a{};
    a.sieve = ctx->d_sieve;
    a.lo = lo;
    a.count = n1;
    a.out = d_out;
    if ((st = launch_range_expand(ctx, a, s))) return st;
    done = n1;
  }
  // Part at or above S: segmented sieve, then Miller-Rabin on the survivors.
  const uint64_t chunk = std::min<uint64_t>(ctx->q.capacity & ~(uint64_t)(kRangeSegInts - 1),
                                            (uint64_t)1 << 30);
  while (done < count) {
    const uint64_t c_lo = lo + done;
    const uint64_t c_n = std::min(count - done, chunk);
    IP_CUDA(cudaMemsetAsync(ctx->q.counters, 0, kQueueCounters * sizeof(uint32_t), s));
    RangeArgs a{};
    a.lo = c_lo;
    a.count = c_n;
    a.out = d_out + done;
    a.primes = ctx->d_base_primes;
    a.nprimes = ctx->d_nprimes;
    a.q64_n = ctx->q.q64_n;
    a.q64_idx = ctx->q.q64_idx;
    a.counters = ctx->q.counters;
    a.q64_cap = (uint32_t)ctx->q.capacity;
    if ((st = launch_range_sieve(ctx, a, s))) return st;
    if ((st = launch_mr(ctx, ctx->q, d_out + done, c_n, s))) return st;
    done += c_n;
  }
  return ISPRIME_OK;
}

}  // namespace ip
