// device_common.cuh -- device routines shared by the plain and batched kernels.
//
// classify_value: the per-element decision of the classify stage (Sec. 1,
// Sec. 6.1.2-6.1.3): n < 2, even, sieve lookup below S, trial division by the
// odd primes 3..p_k without division, and the routing of survivors to the
// 32- or 64-bit Miller-Rabin test.
// rest64_is_prime_warp / bases_pass_warp: the six bases 325 ... 1795265022 of
// Eq. 4 (all, or a subset) for an n >= 2^32 that passed base 2, warp-
// synchronous.  base2_passes_win / base2_passes: the base-2 strong test.
// lucas_warp: the strong Lucas test of the Baillie-PSW option.
// mr32_is_prime: bases {2, 7, 61} for n < 2^32.
#pragma once
#include "arith.cuh"
#include "tables.cuh"

namespace ip {

// Each translation unit keeps its own copy of the constant tables.
static __constant__ TdTable c_td = make_td_table();
static __constant__ BaseTable c_bases = make_base_table();
static __constant__ Td2Table c_td2 = make_td2_table();

enum : int { kComposite = 0, kPrime = 1, kMR64 = 2, kMR32 = 3, kSieveLookup = 4 };

// Bounds checks of the debug build (compiled with IP_DEBUG_CHECKS; see
// isprime_debug_checks).  IP_CHECK(cond, site) guards one queue append,
// queue read or output store: in the debug build a false cond sets the
// site's bit in this translation unit's check word, counts the violation and
// skips the access (no trap); in the production build it is the constant
// true and costs nothing.  IP_CHECK_READER(name) defines the host function
// that reads (and optionally clears) the translation unit's word.
enum : int {
  kChkQ64Front = 0, kChkQ64Back, kChkQ32, kChkOut, kChkQ64Read, kChkQ64b, kChkMrOut, kChkRestRead,
  kChkRestOut, kChkMr32, kChkSmemQueue, kChkBatchOut, kChkRangeQueue, kChkRangeOut, kChkWindow,
  kChkSmallOut, kChkSites
};
#if defined(IP_DEBUG_CHECKS)
static __device__ unsigned int g_ip_check_sites;
static __device__ unsigned long long g_ip_check_count;
__device__ __forceinline__ bool ip_check(bool ok, int site) {
  if (!ok) {
    atomicOr(&g_ip_check_sites, 1u << site);
    atomicAdd(&g_ip_check_count, 1ull);
  }
  return ok;
}
#define IP_CHECK(cond, site) (::ip::ip_check((cond), (site)))
#define IP_CHECK_READER(name)                                                        \
  int name(uint32_t* sites, uint64_t* count, bool reset) {                           \
    unsigned int s = 0;                                                              \
    unsigned long long c = 0;                                                        \
    IP_CUDA(cudaMemcpyFromSymbol(&s, g_ip_check_sites, sizeof s));                   \
    IP_CUDA(cudaMemcpyFromSymbol(&c, g_ip_check_count, sizeof c));                   \
    *sites = s;                                                                      \
    *count = c;                                                                      \
    if (reset) {                                                                     \
      s = 0;                                                                         \
      c = 0;                                                                         \
      IP_CUDA(cudaMemcpyToSymbol(g_ip_check_sites, &s, sizeof s));                   \
      IP_CUDA(cudaMemcpyToSymbol(g_ip_check_count, &c, sizeof c));                   \
    }                                                                                \
    return ISPRIME_OK;                                                               \
  }
#else
#define IP_CHECK(cond, site) (true)
#define IP_CHECK_READER(name)                              \
  int name(uint32_t* sites, uint64_t* count, bool) {       \
    *sites = 0;                                            \
    *count = 0;                                            \
    return ISPRIME_OK;                                     \
  }
#endif

// Double input: finite, >= 0, integral and <= 2^53 (Sec. 8.1) converts
// exactly; anything else is invalid (output 0, counted).
__device__ __forceinline__ bool f64_to_u64(double x, uint64_t* v) {
  const bool ok = (x >= 0.0) && (x <= 9007199254740992.0) && (floor(x) == x);
  *v = ok ? (uint64_t)x : 0ull;
  return ok;
}

constexpr int kWin = 4;
constexpr int kTab = 1 << kWin;

// Chunk sums of n = hi 2^32 + lo modulo 2^k - 1 (see fold_width in tables.cuh);
// each result is below 2^32 and congruent to n modulo 2^k - 1.
__device__ __forceinline__ uint32_t fold_sum32(uint32_t lo, uint32_t hi) {
  const uint64_t s = (uint64_t)lo + hi;  // < 2^33; the carry wraps around
  return (uint32_t)s + (uint32_t)(s >> 32);
}
__device__ __forceinline__ uint32_t fold_sum24(uint32_t lo, uint32_t hi) {
  return (lo & 0xFFFFFFu) + (__funnelshift_r(lo, hi, 24) & 0xFFFFFFu) + (hi >> 16);
}
__device__ __forceinline__ uint32_t fold_sum20(uint32_t lo, uint32_t hi) {
  return (lo & 0xFFFFFu) + (__funnelshift_r(lo, hi, 20) & 0xFFFFFu) + ((hi >> 8) & 0xFFFFFu) +
         (hi >> 28);
}
__device__ __forceinline__ uint32_t fold_sum28(uint32_t lo, uint32_t hi) {
  return (lo & 0xFFFFFFFu) + (__funnelshift_r(lo, hi, 28) & 0xFFFFFFFu) + (hi >> 24);
}

// kNtd >= 0: the trial-division count is a compile-time constant, the loops
// unroll and the inverses and limits become constant operands of the
// multiply and compare instructions.  kNtd < 0: runtime count a.ntd.
// kDefer: an odd n below the sieve limit returns kSieveLookup instead of its
// sieve bit, so that the caller can issue the lookups of several values
// together.  kFold (compile-time kNtd only): the fold level of the 64-bit
// trial division, 0 none, 1 or 2 (fold_width in tables.cuh).
template <int kNtd, typename P, bool kDefer = false, int kFold = 0>
__device__ __forceinline__ int classify_value(uint64_t n, const P& a) {
  if (n < 2) return kComposite;
  if ((n & 1) == 0) return n == 2 ? kPrime : kComposite;
  if (n < a.sieve_limit)
    return kDefer ? kSieveLookup
                  : (int)((__ldg(a.sieve + (n >> 6)) >> ((uint32_t)(n >> 1) & 31u)) & 1u);
  bool hit = false, equal = false;
  const uint32_t ntd = kNtd >= 0 ? (uint32_t)kNtd : a.ntd;
  if constexpr (kNtd != 0) {
    if (n < (1ull << 32)) {
      const uint32_t v = (uint32_t)n;
#pragma unroll
      for (uint32_t i = 0; i < (kNtd >= 0 ? (uint32_t)kNtd : ntd); ++i) {
        hit |= v * c_td.inv32[i] <= c_td.lim32[i];
        equal |= v == c_td.p[i];
      }
    } else if constexpr (kFold == 3 && kNtd == kFoldPrimes) {
      hit = td_pair_divisible(n, c_td.inv32, c_td.lim32);
    } else if constexpr (kFold > 0 && kNtd > 0) {
      const uint32_t lo = (uint32_t)n, hi = (uint32_t)(n >> 32);
      const uint32_t v32 = fold_sum32(lo, hi), v24 = fold_sum24(lo, hi);
      const uint32_t v20 = fold_sum20(lo, hi), v28 = kFold >= 2 ? fold_sum28(lo, hi) : 0u;
#pragma unroll
      for (int i = 0; i < kNtd; ++i) {
        const int k = fold_width(i, kFold);
        const uint32_t v = k == 32 ? v32 : k == 24 ? v24 : k == 20 ? v20 : v28;
        if (k != 0)
          hit |= v * c_td.inv32[i] <= c_td.lim32[i];
        else
          hit |= n * c_td.inv64[i] <= c_td.lim64[i];
      }
    } else {
#pragma unroll
      for (uint32_t i = 0; i < (kNtd >= 0 ? (uint32_t)kNtd : ntd); ++i)
        hit |= n * c_td.inv64[i] <= c_td.lim64[i];
    }
  }
  if (equal) return kPrime;
  if (hit) return kComposite;
  if (n < a.td_square) return kPrime;
  return n < (1ull << 32) ? kMR32 : kMR64;
}

// a^d mod n in Montgomery form by kW-bit fixed windows over the digits of d
// (kW = 4: a table of 16 powers, 14 products to build it and one product
// per four squarings; kW = 3: 8 powers, 6 products, one per three squarings;
// for a 63-bit d that is 89 against 86 Montgomery operations).  tab points
// at this thread's column of the shared table (stride `ld`); nib_warp is the
// warp's largest digit count (leading zero digits select tab[0] = 1).
template <int kImpl, int kW = kWin>
__device__ __forceinline__ uint64_t mont_pow_win(const Mont64& M, uint64_t aR, uint64_t d,
                                                 uint64_t* tab, int ld, int nib_warp = 0) {
  using Ops = MontOps<kImpl>;
  constexpr int kT = 1 << kW;
  tab[0] = M.one;
  tab[ld] = aR;
  uint64_t t = Ops::sqr(aR, M);
  tab[2 * ld] = t;
#pragma unroll
  for (int j = 3; j < kT; ++j) {
    t = Ops::mul(t, aR, M);
    tab[j * ld] = t;
  }
  int nib = (64 - clz64(d) + kW - 1) / kW;  // digits in d (d >= 1)
  if (nib_warp > nib) nib = nib_warp;
  uint64_t x = tab[(int)((d >> (kW * (nib - 1))) & (kT - 1)) * ld];
  for (int k = nib - 2; k >= 0; --k) {
#pragma unroll
    for (int r = 0; r < kW; ++r) x = Ops::sqr(x, M);
    x = Ops::mul(x, tab[(int)((d >> (kW * k)) & (kT - 1)) * ld], M);
  }
  return x;
}

// a^d and b^d mod n at once (two bases, one exponent): the schedule of
// mont_pow_win run on both in one loop, the second table at tb, so that the
// products of one chain overlap the carry chains of the other.  nib_warp is
// the warp's largest digit count (>= this lane's).
template <int kImpl, int kW>
__device__ __forceinline__ void mont_pow_win2(const Mont64& M, uint64_t aR, uint64_t bR, uint64_t d,
                                              uint64_t* ta, uint64_t* tb, int ld, int nib_warp,
                                              uint64_t* xa, uint64_t* xb) {
  using Ops = MontOps<kImpl>;
  constexpr int kT = 1 << kW;
  ta[0] = M.one;
  tb[0] = M.one;
  ta[ld] = aR;
  tb[ld] = bR;
  uint64_t s = Ops::sqr(aR, M), t = Ops::sqr(bR, M);
  ta[2 * ld] = s;
  tb[2 * ld] = t;
#pragma unroll
  for (int j = 3; j < kT; ++j) {
    s = Ops::mul(s, aR, M);
    t = Ops::mul(t, bR, M);
    ta[j * ld] = s;
    tb[j * ld] = t;
  }
  const int nib = nib_warp;
  const int top = (int)((d >> (kW * (nib - 1))) & (kT - 1));
  uint64_t x = ta[top * ld], y = tb[top * ld];
  for (int k = nib - 2; k >= 0; --k) {
#pragma unroll
    for (int r = 0; r < kW; ++r) {
      x = Ops::sqr(x, M);
      y = Ops::sqr(y, M);
    }
    const int dg = (int)((d >> (kW * k)) & (kT - 1));
    x = Ops::mul(x, ta[dg * ld], M);
    y = Ops::mul(y, tb[dg * ld], M);
  }
  *xa = x;
  *xb = y;
}

// Digits of kW bits in d >= 1.
template <int kW>
__device__ __forceinline__ int win_digits(uint64_t d) {
  return (64 - clz64(d) + kW - 1) / kW;
}

// The six bases after base 2 (Eq. 4) for odd n >= 2^32 (no base is 0 mod n),
// warp-synchronous: all 32 lanes call it; the six exponentiations run the
// warp's largest nibble count and every base runs (the inputs are almost all
// primes, which need all six anyway), so the warp never splits.  Lanes with
// valid == false pass any odd n >= 2^32.
template <int kImpl, int kW = kWin>
__device__ __forceinline__ bool rest64_is_prime_warp(uint64_t n, bool valid, uint64_t* tab, int ld) {
  const Mont64 M = mont64_setup(n);
  const uint64_t r2 = mont64_r2<kImpl>(M);
  uint64_t d = n - 1;
  const int s = ctz64(d);
  d >>= s;
  const int nib = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)win_digits<kW>(d));
  bool prime = true;
#pragma unroll 1
  for (int b = 1; b < kNumBases64; ++b) {
    const uint64_t aR = MontOps<kImpl>::mul((uint64_t)c_bases.b64[b], r2, M);
    const uint64_t x = mont_pow_win<kImpl, kW>(M, aR, d, tab, ld, nib);
    prime = prime && sprp_tail64<kImpl>(M, x, s);
    __syncwarp();
  }
  return valid && prime;
}

// rest64_is_prime_warp with the six bases in pairs (mont_pow_win2; tab2 is
// the second table, same stride).
template <int kImpl, int kW>
__device__ __forceinline__ bool rest64_is_prime_warp2(uint64_t n, bool valid, uint64_t* tab,
                                                      uint64_t* tab2, int ld) {
  const Mont64 M = mont64_setup(n);
  const uint64_t r2 = mont64_r2<kImpl>(M);
  uint64_t d = n - 1;
  const int s = ctz64(d);
  d >>= s;
  const int nib = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)win_digits<kW>(d));
  bool prime = true;
#pragma unroll 1
  for (int b = 1; b < kNumBases64; b += 2) {
    const uint64_t aR = MontOps<kImpl>::mul((uint64_t)c_bases.b64[b], r2, M);
    const uint64_t bR = MontOps<kImpl>::mul((uint64_t)c_bases.b64[b + 1], r2, M);
    uint64_t x, y;
    mont_pow_win2<kImpl, kW>(M, aR, bR, d, tab, tab2, ld, nib, &x, &y);
    prime = prime && sprp_tail64<kImpl>(M, x, s);
    __syncwarp();
    prime = prime && sprp_tail64<kImpl>(M, y, s);
    __syncwarp();
  }
  return valid && prime;
}
static_assert((kNumBases64 - 1) % 2 == 0, "the six bases after base 2 pair up");

// The bases of Eq. 4 with indices first .. first + cnt - 1 (first >= 1) for
// an odd n >= 2^32 that passed base 2: true when all pass.  Warp-synchronous
// like rest64_is_prime_warp (all 32 lanes call it with the same cnt, any mix
// of n and first; every exponentiation runs the warp's largest nibble count).
template <int kImpl, int kW = kWin>
__device__ __forceinline__ bool bases_pass_warp(uint64_t n, int first, int cnt, uint64_t* tab,
                                                int ld) {
  const Mont64 M = mont64_setup(n);
  const uint64_t r2 = mont64_r2<kImpl>(M);
  uint64_t d = n - 1;
  const int s = ctz64(d);
  d >>= s;
  const int nib = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)win_digits<kW>(d));
  bool pass = true;
#pragma unroll 1
  for (int k = 0; k < cnt; ++k) {
    const uint64_t aR = MontOps<kImpl>::mul((uint64_t)c_bases.b64[first + k], r2, M);
    pass = pass && sprp_tail64<kImpl>(M, mont_pow_win<kImpl, kW>(M, aR, d, tab, ld, nib), s);
    __syncwarp();
  }
  return pass;
}

// Base 2 with 4-bit windows: T[w] = 2^w R mod n for w < 16 by doublings,
// then per nibble of d four squarings and one multiplication by T[w]; this
// replaces a doubling and a select after every squaring with one
// multiplication every four.  nib_warp (>= this lane's nibble count, the same
// for the whole warp) keeps the loop uniform: leading zero nibbles square the
// Montgomery 1, which stays 1.
template <int kImpl>
__device__ __forceinline__ bool base2_passes_win(uint64_t n, uint64_t* tab, int ld, int nib_warp) {
  using Ops = MontOps<kImpl>;
  const Mont64 M = mont64_setup(n);
  uint64_t d = n - 1;
  const int s = ctz64(d);
  d >>= s;
  uint64_t t = M.one;
  tab[0] = t;
#pragma unroll
  for (int w = 1; w < 16; ++w) {
    t = mod_dbl(t, n);
    tab[w * ld] = t;
  }
  uint64_t e = nib_warp >= 16 ? d : d << (64 - 4 * nib_warp);  // left-aligned exponent
  uint64_t x = tab[(int)(e >> 60) * ld];
  for (int k = 1; k < nib_warp; ++k) {
    e <<= 4;
#pragma unroll
    for (int r = 0; r < 4; ++r) x = Ops::sqr(x, M);
    x = Ops::mul(x, tab[(int)(e >> 60) * ld], M);
  }
  return sprp_tail64<kImpl>(M, x, s);
}

// x 2^w mod n for x < n, 0 <= w <= 15 and odd n >= 2^32, without a
// Montgomery product: x 2^w - q n with the quotient q = floor(x 2^w / n)
// estimated in single precision.  n is normalised (N = n << clz(n), top word
// nt >= 2^31) and x shifted alike (top word xt); then |x/n - xt/nt| < 2^-31,
// the float quotient adds at most 2^-22 (four roundings of a value <= 1), and
// after the exact scaling by 2^w one FMA subtracts 1/32 with an error below
// 2^-9.  So v lies within 2^-6 of t - 1/32 (t = x 2^w / n < 2^15): floor(v) is
// floor(t) or floor(t) - 1, and v < 0 only when floor(t) = 0 (clamped).  The
// remainder x 2^w - q n is then in [0, 2n) and one conditional subtraction of
// n finishes it.  Multiplication by a plain power of two commutes with the
// Montgomery map, so x may be a Montgomery residue.
struct Pow2Red {
  uint32_t sh;   // clz(n) (at most 31)
  float inv;     // 1 / float(top word of n << sh)
  uint32_t rcp;  // min(floor(inv 2^63), 2^32 - 1): 2^63 / nt within a relative 2^-22
};

__device__ __forceinline__ Pow2Red pow2red_setup(uint64_t n) {
  Pow2Red P;
  P.sh = (uint32_t)__clzll((long long)n);
  const uint32_t nt = __funnelshift_l((uint32_t)n, (uint32_t)(n >> 32), P.sh);
  P.inv = __frcp_rn(__uint2float_rn(nt));
  P.rcp = __float2uint_rz(__fmul_rn(P.inv, 9223372036854775808.0f));  // saturates at 2^32 - 1
  return P;
}

// x 2^w - q n for a given estimate q of floor(x 2^w / n) that is exact or one
// less: the remainder is in [0, 2n), and one conditional subtraction ends it.
__device__ __forceinline__ uint64_t pow2_remainder(uint64_t x, uint32_t w, uint64_t n, uint32_t q) {
  const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
  const uint32_t y0 = x0 << w, y1 = __funnelshift_l(x0, x1, w), y2 = __funnelshift_l(x1, 0u, w);
  uint32_t r0, r1, d0, d1, d2;
  asm("{\n\t.reg .u32 pl, ph, sl, sh, r2;\n\t.reg .u64 p, s;\n\t"
      "mul.wide.u32 p, %5, %6;\n\t"
      "mul.wide.u32 s, %5, %7;\n\t"
      "mov.b64 {pl, ph}, p;\n\t"
      "mov.b64 {sl, sh}, s;\n\t"
      "add.cc.u32 ph, ph, sl;\n\t"  // q n = (sh : ph : pl)
      "addc.u32 sh, sh, 0;\n\t"
      "sub.cc.u32 %0, %8, pl;\n\t"  // r = y - q n, in [0, 2n)
      "subc.cc.u32 %1, %9, ph;\n\t"
      "subc.u32 r2, %10, sh;\n\t"
      "sub.cc.u32 %2, %0, %6;\n\t"  // d = r - n
      "subc.cc.u32 %3, %1, %7;\n\t"
      "subc.u32 %4, r2, 0;\n\t"
      "}"
      : "=r"(r0), "=r"(r1), "=r"(d0), "=r"(d1), "=r"(d2)
      : "r"(q), "r"((uint32_t)n), "r"((uint32_t)(n >> 32)), "r"(y0), "r"(y1), "r"(y2));
  return (int32_t)d2 < 0 ? (((uint64_t)r1 << 32) | r0) : (((uint64_t)d1 << 32) | d0);
}

// x 2^w mod n (x < n, w <= 15, odd n >= 2^32) with the quotient estimated in
// integers (base2_window 2): e = floor(xt rcp / 2^32) is (x / n) 2^31 within
// 2^9 + 3 (rcp's relative error 2^-22 gives 2^9, the truncation of x and n to
// their top words 2, the floor 1), so with the bias 2^10 subtracted (clamped
// at 0), q = e' >> (31 - w) is floor(x 2^w / n) or one less: before the
// floor, e' 2^(w - 31) lies at most (2^10 + 2^9 + 3) 2^(w - 31) < 1/32 below
// x 2^w / n and never above it (w <= 15).
__device__ __forceinline__ uint64_t mul_pow2_mod_int(uint64_t x, uint32_t w, uint64_t n,
                                                     const Pow2Red& P) {
  const uint32_t xt = __funnelshift_l((uint32_t)x, (uint32_t)(x >> 32), P.sh);
  const uint32_t e = __umulhi(xt, P.rcp);
  const uint32_t q = (e > 1024u ? e - 1024u : 0u) >> (31u - w);
  return pow2_remainder(x, w, n, q);
}

__device__ __forceinline__ uint64_t mul_pow2_mod(uint64_t x, uint32_t w, uint64_t n,
                                                 const Pow2Red& P) {
  const uint32_t xt = __funnelshift_l((uint32_t)x, (uint32_t)(x >> 32), P.sh);
  const float p2w = __uint_as_float((127u + w) << 23);  // 2^w, exact
  const float v = fmaxf(__fmaf_rn(__fmul_rn(__uint2float_rn(xt), P.inv), p2w, -0.03125f), 0.0f);
  return pow2_remainder(x, w, n, __float2uint_rz(v));
}

// Base 2 with 4-bit windows and no table: per nibble w of d four squarings
// and x 2^w mod n by mul_pow2_mod.  Same warp-uniform schedule as
// base2_passes_win (leading zero nibbles square the Montgomery 1).  n >= 2^32.
template <int kImpl, bool kIntEst = false>
__device__ __forceinline__ bool base2_passes_shift(uint64_t n, int nib_warp) {
  using Ops = MontOps<kImpl>;
  const Mont64 M = mont64_setup(n);
  const Pow2Red P = pow2red_setup(n);
  uint64_t d = n - 1;
  const int s = ctz64(d);
  d >>= s;
  uint64_t e = nib_warp >= 16 ? d : d << (64 - 4 * nib_warp);  // left-aligned exponent
  auto step = [&](uint64_t v, uint32_t w) {
    return kIntEst ? mul_pow2_mod_int(v, w, n, P) : mul_pow2_mod(v, w, n, P);
  };
  uint64_t x = step(M.one, (uint32_t)(e >> 60));
  op_note<kImpl>(2);
  for (int k = 1; k < nib_warp; ++k) {
    e <<= 4;
#pragma unroll
    for (int r = 0; r < 4; ++r) x = Ops::sqr(x, M);
    x = step(x, (uint32_t)(e >> 60));
    op_note<kImpl>(2);
  }
  return sprp_tail64<kImpl>(M, x, s);
}

// Base 2 for two values at once (odd na, nb >= 2^32), the schedule of
// base2_passes_shift run on both in one loop: the two exponentiations are
// independent, so the multiplies of one overlap the carry chains of the
// other.  nib_warp covers both values of every lane of the warp.  The
// strong-test tails run until both values are decided.
template <int kImpl>
__device__ __forceinline__ void base2_passes_shift_x2(uint64_t na, uint64_t nb, int nib_warp,
                                                      bool* pass_a, bool* pass_b) {
  using Ops = MontOps<kImpl>;
  const Mont64 Ma = mont64_setup(na), Mb = mont64_setup(nb);
  const Pow2Red Pa = pow2red_setup(na), Pb = pow2red_setup(nb);
  uint64_t da = na - 1, db = nb - 1;
  const int sa = ctz64(da), sb = ctz64(db);
  da >>= sa;
  db >>= sb;
  uint64_t ea = nib_warp >= 16 ? da : da << (64 - 4 * nib_warp);
  uint64_t eb = nib_warp >= 16 ? db : db << (64 - 4 * nib_warp);
  uint64_t xa = mul_pow2_mod(Ma.one, (uint32_t)(ea >> 60), na, Pa);
  op_note<kImpl>(2);
  uint64_t xb = mul_pow2_mod(Mb.one, (uint32_t)(eb >> 60), nb, Pb);
  op_note<kImpl>(2);
  for (int k = 1; k < nib_warp; ++k) {
    ea <<= 4;
    eb <<= 4;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      xa = Ops::sqr(xa, Ma);
      xb = Ops::sqr(xb, Mb);
    }
    xa = mul_pow2_mod(xa, (uint32_t)(ea >> 60), na, Pa);
    op_note<kImpl>(2);
    xb = mul_pow2_mod(xb, (uint32_t)(eb >> 60), nb, Pb);
    op_note<kImpl>(2);
  }
  // a passes when a^d = +-1, or a^(d 2^r) = -1 for some 1 <= r < s; a value
  // of 1 after a squaring ends the test (it stays 1)
  bool pa = xa == Ma.one || xa == Ma.mone, pb = xb == Mb.one || xb == Mb.mone;
  bool done_a = pa || sa <= 1, done_b = pb || sb <= 1;
  for (int r = 1; !(done_a && done_b); ++r) {
    if (!done_a) {
      xa = Ops::sqr(xa, Ma);
      pa = xa == Ma.mone;
      done_a = pa || xa == Ma.one || r + 1 >= sa;
    }
    if (!done_b) {
      xb = Ops::sqr(xb, Mb);
      pb = xb == Mb.mone;
      done_b = pb || xb == Mb.one || r + 1 >= sb;
    }
  }
  *pass_a = pa;
  *pass_b = pb;
}

// Number of 4-bit nibbles of the odd part of n - 1.
__device__ __forceinline__ int base2_nibbles(uint64_t n) {
  uint64_t d = n - 1;
  d >>= ctz64(d);
  return (64 - clz64(d) + 3) >> 2;
}

// Warp-synchronous strong Lucas test: all 32 lanes of a converged warp call
// it (lanes with valid == false pass any odd n and ignore the result).  The
// D search advances in lock step until every lane has its D, and the ladder
// runs the warp's largest bit count, so the lanes never split into groups
// that would run the ladder one after another.
template <int kImpl>
__device__ __forceinline__ bool lucas_warp(uint64_t n, bool valid) {
  int32_t D = 5;
  int k = 0, st = (n == ~0ull) ? 1 : -1;
  while (__any_sync(0xFFFFFFFFu, st < 0)) {
    if (st < 0) st = lucas_next_D(n, &D, &k);
  }
  const int nb = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)lucas_bits(n));
  const bool prime = lucas_ladder<kImpl>(n, st ? 5 : D, nb);
  return valid && st == 0 && prime;
}

// Base 2 for odd n >= 2^32.
template <int kImpl>
__device__ __forceinline__ bool base2_passes(uint64_t n) {
  const Mont64 M = mont64_setup(n);
  uint64_t d = n - 1;
  const int s = ctz64(d);
  d >>= s;
  return sprp2_64<kImpl>(M, d, s);
}

// Bases {2, 7, 61} for odd n < 2^32 (exact below 4,759,123,141).
__device__ __forceinline__ bool mr32_is_prime(uint32_t n) {
  const Mont32 M = mont32_setup(n);
  uint32_t d = n - 1;
  const int s = ctz32(d);
  d >>= s;
#pragma unroll 1
  for (int b = 0; b < kNumBases32; ++b) {
    const uint32_t a = c_bases.b32[b] % n;
    if (a == 0) continue;  // base divisible by n: skipped (n is 7 or 61 here)
    if (!sprp32(M, a, d, s)) return false;
  }
  return true;
}

}  // namespace ip
