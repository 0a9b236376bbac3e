// sieve.cu -- device-resident odd-only sieve of Eratosthenes.
//
// The paper's long-array path computes every prime up to the array maximum
// and then looks elements up (Sec. 6.1.3, which minimises the number of
// divisions); the sieve itself is described in Sec. 1.  Here the sieve is
// built once per context on the GPU for [0, S) and kept resident, so a
// lookup is one bit read.
//
// Layout: bit j (word j/32, bit j%32) stands for the odd number 2j+1, so S
// values take S/16 bytes.  Build: one block sieves the odd primes below 2^16
// (enough for S <= 2^32); then one block per segment of SEG_WORDS words
// crosses off multiples in shared memory and writes the segment with
// coalesced 16-byte stores.
#include "internal.h"

namespace ip {

constexpr int kBaseThreads = 1024;
constexpr int kBaseWords = 1024;  // 32768 bits: odd numbers below 65536
constexpr int kSegWords = 8192;   // 32 KiB of shared memory per segment
constexpr int kSegThreads = 512;
constexpr int kNumSmallPrimes = 10;  // 3..31: crossed off by word masks
__constant__ uint32_t c_small_primes[kNumSmallPrimes] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};

// Odd primes below 2^16 in ascending order, and their count.
__global__ void __launch_bounds__(kBaseThreads) sieve_base_kernel(uint32_t* primes, uint32_t* count) {
  __shared__ uint32_t bits[kBaseWords];
  __shared__ uint32_t warp_tot[kBaseThreads / 32];
  const int tid = threadIdx.x;
  bits[tid] = 0xFFFFFFFFu;
  __syncthreads();
  if (tid == 0) bits[0] &= ~1u;  // 1 is not prime
  __syncthreads();
  for (uint32_t p = 3; p * p < 65536u; p += 2) {
    const uint32_t jp = p >> 1;
    const bool isp = (bits[jp >> 5] >> (jp & 31)) & 1u;  // p's own bit is never cleared here
    if (isp) {
      for (uint32_t j = ((p * p) >> 1) + tid * p; j < kBaseWords * 32u; j += p * kBaseThreads)
        atomicAnd(&bits[j >> 5], ~(1u << (j & 31)));
    }
    __syncthreads();
  }
  // Compact the set bits in ascending order: block-wide exclusive scan of
  // per-word popcounts.
  const uint32_t w = bits[tid];
  const uint32_t c = __popc(w);
  const int lane = tid & 31, warp = tid >> 5;
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = warp_tot[lane];
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t v = __shfl_up_sync(0xFFFFFFFFu, ti, o);
      if (lane >= o) ti += v;
    }
    warp_tot[lane] = ti - t;  // exclusive prefix of warp totals
    if (lane == 31) *count = ti;
  }
  __syncthreads();
  uint32_t pos = warp_tot[warp] + incl - c;
  uint32_t ww = w;
  while (ww) {
    int b = __ffs(ww) - 1;
    ww &= ww - 1;
    primes[pos++] = 2u * (32u * (uint32_t)tid + (uint32_t)b) + 1u;
  }
}

__device__ __forceinline__ void clear_bit(uint32_t* seg, uint32_t j) {
  atomicAnd(&seg[j >> 5], ~(1u << (j & 31)));
}

// One block per segment of kSegWords words.  J0 = first bit index of the
// segment; bit j <-> 2j+1.  Multiples of p that are odd sit at bits
// j = (p-1)/2 (mod p); crossing starts at p^2, so primes keep their bits.
__global__ void __launch_bounds__(kSegThreads)
    sieve_segment_kernel(uint32_t* bitmap, uint64_t total_words, const uint32_t* primes,
                         const uint32_t* nprimes_ptr) {
  __shared__ __align__(16) uint32_t seg[kSegWords];
  const uint32_t tid = threadIdx.x;
  const uint64_t w0 = (uint64_t)blockIdx.x * kSegWords;
  const uint64_t J0 = w0 * 32;
  const uint64_t J1 = J0 + (uint64_t)kSegWords * 32;  // exclusive
  const uint64_t vmax = 2 * J1 - 1;                   // largest odd value in the segment

  // 1) small primes by per-word masks (several bits per word)
  for (uint32_t w = tid; w < kSegWords; w += kSegThreads) {
    const uint32_t jw = (uint32_t)(J0 + 32ull * w);  // < 2^31 because S <= 2^32
    uint32_t m = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < kNumSmallPrimes; ++k) {
      const uint32_t p = c_small_primes[k];
      const uint32_t r = (p - 1) >> 1;
      const uint32_t jm = jw % p;
      uint32_t off = (r + p - jm) % p;  // first bit in this word with j = r (mod p)
      for (uint32_t b = off; b < 32; b += p) {
        // keep p itself (j = r): crossing starts at p^2
        if (jw + b != r) m &= ~(1u << b);
      }
    }
    seg[w] = m;
  }
  __syncthreads();
  if (blockIdx.x == 0 && tid == 0) seg[0] &= ~1u;  // 1 is not prime
  __syncthreads();

  // 2) larger primes: one warp per prime while a prime has many multiples in
  //    the segment, one thread per prime beyond that.
  const uint32_t np = *nprimes_ptr;
  const uint32_t lane = tid & 31, warp = tid >> 5, nwarps = kSegThreads / 32;
  constexpr uint32_t kWarpPrimeLimit = 4096;
  uint32_t i_split = kNumSmallPrimes;
  // index of the first prime >= kWarpPrimeLimit (primes are sorted; at most 564 below 4096)
  {
    uint32_t lo = kNumSmallPrimes, hi = np;
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (primes[mid] < kWarpPrimeLimit) lo = mid + 1; else hi = mid;
    }
    i_split = lo;
  }
  for (uint32_t i = kNumSmallPrimes + warp; i < i_split; i += nwarps) {
    const uint64_t p = primes[i];
    if (p * p > vmax) break;
    const uint64_t r = (p - 1) >> 1;
    uint64_t start = (p * p - 1) >> 1;
    if (start < J0) start = J0;
    const uint64_t rem = (start - r) % p;
    const uint64_t first = rem ? start + (p - rem) : start;
    for (uint64_t j = first + lane * p; j < J1; j += 32 * p) clear_bit(seg, (uint32_t)(j - J0));
  }
  for (uint32_t i = i_split + tid; i < np; i += kSegThreads) {
    const uint64_t p = primes[i];
    if (p * p > vmax) break;
    const uint64_t r = (p - 1) >> 1;
    uint64_t start = (p * p - 1) >> 1;
    if (start < J0) start = J0;
    const uint64_t rem = (start - r) % p;
    const uint64_t first = rem ? start + (p - rem) : start;
    for (uint64_t j = first; j < J1; j += p) clear_bit(seg, (uint32_t)(j - J0));
  }
  __syncthreads();

  // 3) coalesced 16-byte stores of the segment
  const uint4* s4 = reinterpret_cast<const uint4*>(seg);
  uint4* g4 = reinterpret_cast<uint4*>(bitmap + w0);
  const uint64_t words_left = total_words - w0;
  const uint32_t nw = words_left < (uint64_t)kSegWords ? (uint32_t)words_left : (uint32_t)kSegWords;
  for (uint32_t v = tid; v < nw / 4; v += kSegThreads) g4[v] = s4[v];
  for (uint32_t w = (nw / 4) * 4 + tid; w < nw; w += kSegThreads) bitmap[w0 + w] = seg[w];
}

__global__ void sieve_count_kernel(const uint32_t* bitmap, uint64_t total_words,
                                   unsigned long long* out) {
  uint64_t acc = 0;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total_words;
       w += (uint64_t)gridDim.x * blockDim.x)
    acc += __popc(bitmap[w]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

// The odd primes below 2^16 and their count, kept on the device by every
// context (the segmented sieves of sieve_build and of range.cu use them).
int ensure_base_primes(isprime_ctx* ctx, cudaStream_t s) {
  if (ctx->d_base_primes) return ISPRIME_OK;
  IP_CUDA(cudaMalloc(&ctx->d_base_primes, 8192 * sizeof(uint32_t)));
  IP_CUDA(cudaMalloc(&ctx->d_nprimes, sizeof(uint32_t)));
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_SIEVE_BASE, s, &tl);
  if (st) return st;
  sieve_base_kernel<<<1, kBaseThreads, 0, s>>>(ctx->d_base_primes, ctx->d_nprimes);
  if ((st = launch_end(ctx, s, &tl, "sieve_base_kernel"))) return st;
  IP_CUDA(cudaMemcpyAsync(&ctx->n_base_primes, ctx->d_nprimes, sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, s));
  IP_CUDA(cudaStreamSynchronize(s));
  return ISPRIME_OK;
}

int sieve_build(isprime_ctx* ctx, cudaStream_t s) {
  int st = ensure_base_primes(ctx, s);
  if (st || ctx->sieve_limit == 0) return st;
  const uint64_t total_words = ctx->sieve_limit / 64;
  const uint64_t nseg = (total_words + kSegWords - 1) / kSegWords;
  TimedLaunch tl;
  if ((st = launch_begin(ctx, ISPRIME_K_SIEVE_SEGMENT, s, &tl))) return st;
  sieve_segment_kernel<<<(unsigned)nseg, kSegThreads, 0, s>>>(ctx->d_sieve, total_words,
                                                               ctx->d_base_primes, ctx->d_nprimes);
  if ((st = launch_end(ctx, s, &tl, "sieve_segment_kernel"))) return st;
  IP_CUDA(cudaStreamSynchronize(s));
  return ISPRIME_OK;
}

int sieve_count(isprime_ctx* ctx, cudaStream_t s, uint64_t* d_out) {
  if (ctx->sieve_limit == 0) return ISPRIME_OK;
  const uint64_t total_words = ctx->sieve_limit / 64;
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_SIEVE_COUNT, s, &tl);
  if (st) return st;
  sieve_count_kernel<<<ctx->sm_count * 4, 256, 0, s>>>(ctx->d_sieve, total_words,
                                                        reinterpret_cast<unsigned long long*>(d_out));
  return launch_end(ctx, s, &tl, "sieve_count_kernel");
}

}  // namespace ip
