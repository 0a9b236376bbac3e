// arith.cuh -- modular arithmetic for the primality kernels (sm_103a).
//
// The paper builds Miller-Rabin on three overflow-free helpers: ModAdd,
// ModMultiply and ModExp (Sec. 2.2-2.4).  On the GPU the same results come
// from Montgomery arithmetic: a*b*2^-64 mod n from two 64x64->128 products
// (IMAD chains on the integer pipe), no division on the hot path, and a
// modular doubling for the base-2 test instead of a multiplication.
//
// Every function is __host__ __device__ so that the host-side unit test can
// check the same source against exact big-integer arithmetic; the device
// build uses the __umul64hi intrinsic, the host build a 128-bit product.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define IP_HD __host__ __device__ __forceinline__
#else
#define IP_HD inline
#endif

namespace ip {

IP_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

IP_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

IP_HD int clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return __builtin_clzll(x);
#endif
}

IP_HD int clz32(uint32_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clz((int)x);
#else
  return __builtin_clz(x);
#endif
}

IP_HD int ctz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __ffsll((long long)x) - 1;
#else
  return __builtin_ctzll(x);
#endif
}

IP_HD int ctz32(uint32_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __ffs((int)x) - 1;
#else
  return __builtin_ctz(x);
#endif
}

// n^-1 mod 2^64 for odd n by Newton-Hensel lifting x <- x(2 - n x); the seed
// (3n) xor 2 is correct to 5 bits, each step doubles the correct bits.
IP_HD uint64_t inv64(uint64_t n) {
  uint64_t x = (3 * n) ^ 2;
  x *= 2 - n * x;
  x *= 2 - n * x;
  x *= 2 - n * x;
  x *= 2 - n * x;
  return x;
}

IP_HD uint32_t inv32(uint32_t n) {
  uint32_t x = (3 * n) ^ 2;
  x *= 2 - n * x;
  x *= 2 - n * x;
  x *= 2 - n * x;
  return x;
}

// ---------------------------------------------------------------------------
// 64-bit Montgomery arithmetic, R = 2^64, odd modulus n < 2^64.
// Values in Montgomery form are xR mod n, fully reduced to [0, n).
// ---------------------------------------------------------------------------
struct Mont64 {
  uint64_t n;     // modulus (odd)
  uint64_t ninv;  // n^-1 mod 2^64
  uint64_t one;   // R mod n      (Montgomery form of 1)
  uint64_t mone;  // n - one      (Montgomery form of n-1)
};

// REDC of the 128-bit t = a*b: with m = lo(t) * n^-1 mod 2^64 the low words
// of t and m*n agree, so (t - m n) / 2^64 = hi(t) - hi(m n), in (-n, n).
IP_HD uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t n, uint64_t ninv) {
  uint64_t lo = a * b;
  uint64_t hi = mulhi64(a, b);
  uint64_t m = lo * ninv;
  uint64_t mh = mulhi64(m, n);
  uint64_t r = hi - mh;
  return (hi < mh) ? r + n : r;
}

IP_HD uint64_t mont_sqr(uint64_t a, uint64_t n, uint64_t ninv) {
  return mont_mul(a, a, n, ninv);
}

// 2x mod n for x < n (ModAdd of x to itself, Sec. 2.2): if 2x overflows 64
// bits it is certainly >= n, and the wrapped difference is exact.
IP_HD uint64_t mod_dbl(uint64_t x, uint64_t n) {
  uint64_t y = x << 1;
  return ((int64_t)x < 0 || y >= n) ? y - n : y;
}

IP_HD Mont64 mont64_setup(uint64_t n) {
  Mont64 m;
  m.n = n;
  m.ninv = inv64(n);
  // 2^64 mod n: for n > 2^63 it is 2^64 - n, otherwise reduce (0 - n) mod n.
  m.one = ((int64_t)n < 0) ? (0 - n) : (0 - n) % n;
  m.mone = n - m.one;
  return m;
}

// R^2 mod n from R mod n: 8 doublings give R 2^8; each Montgomery squaring
// maps R 2^k to R 2^(2k): 2^8 -> 2^16 -> 2^32 -> 2^64.
IP_HD uint64_t mont64_r2(const Mont64& M) {
  uint64_t x = M.one;
#pragma unroll
  for (int i = 0; i < 8; ++i) x = mod_dbl(x, M.n);
  x = mont_sqr(x, M.n, M.ninv);
  x = mont_sqr(x, M.n, M.ninv);
  x = mont_sqr(x, M.n, M.ninv);
  return x;
}

// Strong probable-prime test to base 2 (Sec. 2.1), n odd, n > 2.
// 2^d by left-to-right binary exponentiation where "multiply by the base"
// is a modular doubling.
IP_HD bool sprp2_64(const Mont64& M, uint64_t d, int s) {
  const uint64_t n = M.n, ninv = M.ninv;
  int top = 63 - clz64(d);
  uint64_t x = mod_dbl(M.one, n);  // the leading 1 bit: 2 in Montgomery form
  for (int b = top - 1; b >= 0; --b) {
    x = mont_sqr(x, n, ninv);
    uint64_t y = mod_dbl(x, n);
    x = ((d >> b) & 1) ? y : x;
  }
  if (x == M.one || x == M.mone) return true;
  for (int r = 1; r < s; ++r) {
    x = mont_sqr(x, n, ninv);
    if (x == M.mone) return true;
    if (x == M.one) return false;
  }
  return false;
}

// Finishes a strong test once x = a^d (Montgomery form) is known.
IP_HD bool sprp_tail64(const Mont64& M, uint64_t x, int s) {
  if (x == M.one || x == M.mone) return true;
  for (int r = 1; r < s; ++r) {
    x = mont_sqr(x, M.n, M.ninv);
    if (x == M.mone) return true;
    if (x == M.one) return false;
  }
  return false;
}

// a^d for a base a < n given in Montgomery form (aR), plain left-to-right
// binary exponentiation (host reference for the windowed device kernels).
IP_HD uint64_t mont_pow_binary(const Mont64& M, uint64_t aR, uint64_t d) {
  uint64_t x = M.one;
  for (int b = 63 - clz64(d); b >= 0; --b) {
    x = mont_sqr(x, M.n, M.ninv);
    if ((d >> b) & 1) x = mont_mul(x, aR, M.n, M.ninv);
  }
  return x;
}

// ---------------------------------------------------------------------------
// 32-bit Montgomery arithmetic, R = 2^32, odd modulus n < 2^32.
// ---------------------------------------------------------------------------
struct Mont32 {
  uint32_t n, ninv, one, mone;
};

IP_HD uint32_t mont_mul32(uint32_t a, uint32_t b, uint32_t n, uint32_t ninv) {
  uint64_t t = (uint64_t)a * b;
  uint32_t m = (uint32_t)t * ninv;
  uint32_t mh = mulhi32(m, n);
  uint32_t hi = (uint32_t)(t >> 32);
  uint32_t r = hi - mh;
  return (hi < mh) ? r + n : r;
}

IP_HD uint32_t mod_dbl32(uint32_t x, uint32_t n) {
  uint32_t y = x << 1;
  return ((int32_t)x < 0 || y >= n) ? y - n : y;
}

IP_HD Mont32 mont32_setup(uint32_t n) {
  Mont32 m;
  m.n = n;
  m.ninv = inv32(n);
  m.one = (uint32_t)((0x100000000ULL) % n);
  m.mone = n - m.one;
  return m;
}

// Strong test of odd n < 2^32 to base a (1 < a < n).  Base 2 multiplies by
// doubling; other bases enter Montgomery form as a*2^32 mod n.
IP_HD bool sprp32(const Mont32& M, uint32_t a, uint32_t d, int s) {
  const uint32_t n = M.n, ninv = M.ninv;
  uint32_t x;
  int top = 31 - clz32(d);
  if (a == 2) {
    x = mod_dbl32(M.one, n);
    for (int b = top - 1; b >= 0; --b) {
      x = mont_mul32(x, x, n, ninv);
      uint32_t y = mod_dbl32(x, n);
      x = ((d >> b) & 1) ? y : x;
    }
  } else {
    uint32_t aR = (uint32_t)(((uint64_t)a << 32) % n);
    x = aR;
    for (int b = top - 1; b >= 0; --b) {
      x = mont_mul32(x, x, n, ninv);
      uint32_t y = mont_mul32(x, aR, n, ninv);
      x = ((d >> b) & 1) ? y : x;
    }
  }
  if (x == M.one || x == M.mone) return true;
  for (int r = 1; r < s; ++r) {
    x = mont_mul32(x, x, n, ninv);
    if (x == M.mone) return true;
    if (x == M.one) return false;
  }
  return false;
}

}  // namespace ip
