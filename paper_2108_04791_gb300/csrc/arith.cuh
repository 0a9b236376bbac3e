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

#include "tables.cuh"

#if defined(__CUDACC__)
#define IP_HD __host__ __device__ __forceinline__
#else
#define IP_HD inline
#include <math.h>
#endif
// Loop unrolling hint for functions compiled for both sides: the device pass
// takes it, the host compiler does not see it.
#if defined(__CUDA_ARCH__)
#define IP_UNROLL _Pragma("unroll")
#else
#define IP_UNROLL
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
  uint64_t ninv;  // n^-1 mod 2^64 (128-bit-product REDC)
  uint32_t q;     // -n^-1 mod 2^32 (word-level REDC)
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

// Squaring in the same 128-bit form with the cross product computed once:
// a^2 = a0^2 + 2 a0 a1 2^32 + a1^2 2^64 (three wide products instead of
// four); the REDC is the one of mont_mul.
IP_HD uint64_t mont_sqr_h(uint64_t a, uint64_t n, uint64_t ninv) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint64_t L = (uint64_t)a0 * a0;
  const uint64_t X = (uint64_t)a0 * a1;
  const uint64_t Y = (uint64_t)a1 * a1;
  const uint64_t lo = L + (X << 33);
  const uint64_t hi = Y + (X >> 31) + (lo < L);
  const uint64_t m = lo * ninv;
  const uint64_t mh = mulhi64(m, n);
  const uint64_t r = hi - mh;
  return (hi < mh) ? r + n : r;
}

#if defined(__CUDACC__)
// The 128-bit form with the REDC done word by word in PTX carry chains:
// t = a*b from the compiler's 64-bit products, then two rounds of
// m = t_i q mod 2^32, t += m n 2^(32 i) (q = -n^-1 mod 2^32).
__device__ __forceinline__ uint64_t mont_mul_p(uint64_t a, uint64_t b, uint64_t n, uint32_t q) {
  const uint64_t lo = a * b;
  const uint64_t hi = __umul64hi(a, b);
  uint32_t t0 = (uint32_t)lo, t1 = (uint32_t)(lo >> 32), t2 = (uint32_t)hi, t3 = (uint32_t)(hi >> 32);
  uint32_t t4;
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  asm("{\n\t.reg .u32 mm;\n\t"
      "mul.lo.u32      mm, %0, %7;\n\t"
      "mad.lo.cc.u32   %0, mm, %5, %0;\n\t"
      "madc.lo.cc.u32  %1, mm, %6, %1;\n\t"
      "addc.cc.u32     %2, %2, 0;\n\t"
      "addc.cc.u32     %3, %3, 0;\n\t"
      "addc.u32        %4, 0, 0;\n\t"
      "mad.hi.cc.u32   %1, mm, %5, %1;\n\t"
      "madc.hi.cc.u32  %2, mm, %6, %2;\n\t"
      "addc.cc.u32     %3, %3, 0;\n\t"
      "addc.u32        %4, %4, 0;\n\t"
      "mul.lo.u32      mm, %1, %7;\n\t"
      "mad.lo.cc.u32   %1, mm, %5, %1;\n\t"
      "madc.lo.cc.u32  %2, mm, %6, %2;\n\t"
      "addc.cc.u32     %3, %3, 0;\n\t"
      "addc.u32        %4, %4, 0;\n\t"
      "mad.hi.cc.u32   %2, mm, %5, %2;\n\t"
      "madc.hi.cc.u32  %3, mm, %6, %3;\n\t"
      "addc.u32        %4, %4, 0;\n\t}"
      : "+r"(t0), "+r"(t1), "+r"(t2), "+r"(t3), "=r"(t4)
      : "r"(n0), "r"(n1), "r"(q));
  const uint64_t r = ((uint64_t)t3 << 32) | t2;
  return (t4 != 0 || r >= n) ? r - n : r;
}
#endif

#if defined(__CUDACC__)
// The 128-bit form in 32-bit words as PTX, so that each partial product is
// one wide multiply and each sum one add with carry (inputs a, b < n, odd n):
//   a b       = p00 + (p01 + p10) 2^32 + p11 2^64        4 wide products
//   m         = lo64(a b) n^-1 mod 2^64                 1 wide + 2 low products
//   hi64(m n) = q11 + hi(q01) + hi(q10) + c1 + c         3 wide products
// with q_ij = m_i n_j and c1 the carry of lo(q01) + lo(q10) = sl.  The high
// word of m0 n0 is never formed: lo64(m n) = lo64(a b), so bits 32..63 of
// m n are t1 (bits 32..63 of a b), and the carry that word adds at bit 64 is
// c = [sl > t1].  c enters as the borrow of t1 - sl in the subtraction
// r = hi64(a b) - hi64(m n), and n is added back when r < 0.
#define IP_MONT_C_DECL                                                  \
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);            \
  const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);            \
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);            \
  const uint32_t i0 = (uint32_t)ninv, i1 = (uint32_t)(ninv >> 32);      \
  uint32_t r0, r1;
// Operands: %0 %1 result words; %2 %3 a; %4 %5 b; %6 %7 n; %8 %9 n^-1.
#define IP_MONT_C_REGS                                                          \
  ".reg .u32 p00l, p00h, p01l, p01h, p10l, p10h, p11l, p11h, t1, t2, t3;\n\t" \
  ".reg .u32 m0, m1, q01l, q01h, q10l, q10h, q11l, q11h, sl, x, y, bo;\n\t"   \
  ".reg .u64 w;\n\t"
// After p00, p01 and p10: the rest of a b, then m, hi64(m n) and r.
#define IP_MONT_C_TAIL                                                          \
  /* p11 and t = a b = t3:t2:t1:p00l */                                         \
  "mul.wide.u32 w, %3, %5;\n\t"                                                 \
  "mov.b64 {p11l, p11h}, w;\n\t"                                                \
  "add.cc.u32 t1, p00h, p01l;\n\t"                                              \
  "addc.cc.u32 t2, p01h, p11l;\n\t"                                             \
  "addc.u32 t3, p11h, 0;\n\t"                                                   \
  "add.cc.u32 t1, t1, p10l;\n\t"                                                \
  "addc.cc.u32 t2, t2, p10h;\n\t"                                               \
  "addc.u32 t3, t3, 0;\n\t"                                                     \
  /* m = (t1:p00l) n^-1 mod 2^64 */                                             \
  "mul.wide.u32 w, p00l, %8;\n\t"                                               \
  "mov.b64 {m0, m1}, w;\n\t"                                                    \
  "mad.lo.u32 m1, p00l, %9, m1;\n\t"                                            \
  "mad.lo.u32 m1, t1, %8, m1;\n\t"                                              \
  /* q01, q10, q11; (y:x) = q11 + hi(q01) + hi(q10) + c1 */                      \
  "mul.wide.u32 w, m0, %7;\n\t"                                                 \
  "mov.b64 {q01l, q01h}, w;\n\t"                                                \
  "mul.wide.u32 w, m1, %6;\n\t"                                                 \
  "mov.b64 {q10l, q10h}, w;\n\t"                                                \
  "mul.wide.u32 w, m1, %7;\n\t"                                                 \
  "mov.b64 {q11l, q11h}, w;\n\t"                                                \
  "add.cc.u32 sl, q01l, q10l;\n\t"                                              \
  "addc.cc.u32 x, q11l, q01h;\n\t"                                              \
  "addc.u32 y, q11h, 0;\n\t"                                                    \
  "add.cc.u32 x, x, q10h;\n\t"                                                  \
  "addc.u32 y, y, 0;\n\t"                                                       \
  /* r = (t3:t2) - (y:x) - c, c = borrow of t1 - sl; + n if negative */         \
  "sub.cc.u32 bo, t1, sl;\n\t"                                                  \
  "subc.cc.u32 %0, t2, x;\n\t"                                                  \
  "subc.cc.u32 %1, t3, y;\n\t"                                                  \
  "subc.u32 bo, 0, 0;\n\t"                                                      \
  "and.b32 x, bo, %6;\n\t"                                                      \
  "and.b32 y, bo, %7;\n\t"                                                      \
  "add.cc.u32 %0, %0, x;\n\t"                                                   \
  "addc.u32 %1, %1, y;\n\t"
#define IP_MONT_C_OPERANDS                                                      \
  : "=r"(r0), "=r"(r1)                                                          \
  : "r"(a0), "r"(a1), "r"(b0), "r"(b1), "r"(n0), "r"(n1), "r"(i0), "r"(i1)

__device__ __forceinline__ uint64_t mont_mul_c(uint64_t a, uint64_t b, uint64_t n, uint64_t ninv) {
  IP_MONT_C_DECL
  asm("{\n\t" IP_MONT_C_REGS
      "mul.wide.u32 w, %2, %4;\n\t"
      "mov.b64 {p00l, p00h}, w;\n\t"
      "mul.wide.u32 w, %2, %5;\n\t"
      "mov.b64 {p01l, p01h}, w;\n\t"
      "mul.wide.u32 w, %3, %4;\n\t"
      "mov.b64 {p10l, p10h}, w;\n\t"
      IP_MONT_C_TAIL "}" IP_MONT_C_OPERANDS);
  return ((uint64_t)r1 << 32) | r0;
}

// Squaring: b = a, and the cross product a0 a1 serves as both p01 and p10.
__device__ __forceinline__ uint64_t mont_sqr_c(uint64_t a, uint64_t n, uint64_t ninv) {
  const uint64_t b = a;
  IP_MONT_C_DECL
  asm("{\n\t" IP_MONT_C_REGS
      "mul.wide.u32 w, %2, %4;\n\t"
      "mov.b64 {p00l, p00h}, w;\n\t"
      "mul.wide.u32 w, %2, %5;\n\t"
      "mov.b64 {p01l, p01h}, w;\n\t"
      "mov.u32 p10l, p01l;\n\t"
      "mov.u32 p10h, p01h;\n\t"
      IP_MONT_C_TAIL "}" IP_MONT_C_OPERANDS);
  return ((uint64_t)r1 << 32) | r0;
}
// Formulation 9: formulation 6 with the final "+ n when negative" done on the
// multiply pipe: the borrow becomes b in {0, 1} and r + b n is two
// multiply-adds with carry (mad.lo.cc / madc.lo) instead of two ANDs and two
// adds on the ALU pipe.  The arithmetic is the same; only the pipe that does
// the correction changes (for kernels whose ALU pipe is the busier one).
#define IP_MONT_E_TAIL(prefix)                                                  \
  prefix                                                                        \
  "sub.cc.u32 bo, t1, sl;\n\t"                                                  \
  "subc.cc.u32 %0, t2, x;\n\t"                                                  \
  "subc.cc.u32 %1, t3, y;\n\t"                                                  \
  "subc.u32 bo, 0, 0;\n\t"                                                      \
  "and.b32 bo, bo, 1;\n\t"                                                      \
  "mad.lo.cc.u32 %0, bo, %6, %0;\n\t"                                           \
  "madc.lo.u32 %1, bo, %7, %1;\n\t"
#define IP_MONT_E_BODY                                                          \
  /* p11 and t = a b = t3:t2:t1:p00l */                                         \
  "mul.wide.u32 w, %3, %5;\n\t"                                                 \
  "mov.b64 {p11l, p11h}, w;\n\t"                                                \
  "add.cc.u32 t1, p00h, p01l;\n\t"                                              \
  "addc.cc.u32 t2, p01h, p11l;\n\t"                                             \
  "addc.u32 t3, p11h, 0;\n\t"                                                   \
  "add.cc.u32 t1, t1, p10l;\n\t"                                                \
  "addc.cc.u32 t2, t2, p10h;\n\t"                                               \
  "addc.u32 t3, t3, 0;\n\t"                                                     \
  "mul.wide.u32 w, p00l, %8;\n\t"                                               \
  "mov.b64 {m0, m1}, w;\n\t"                                                    \
  "mad.lo.u32 m1, p00l, %9, m1;\n\t"                                            \
  "mad.lo.u32 m1, t1, %8, m1;\n\t"                                              \
  "mul.wide.u32 w, m0, %7;\n\t"                                                 \
  "mov.b64 {q01l, q01h}, w;\n\t"                                                \
  "mul.wide.u32 w, m1, %6;\n\t"                                                 \
  "mov.b64 {q10l, q10h}, w;\n\t"                                                \
  "mul.wide.u32 w, m1, %7;\n\t"                                                 \
  "mov.b64 {q11l, q11h}, w;\n\t"                                                \
  "add.cc.u32 sl, q01l, q10l;\n\t"                                              \
  "addc.cc.u32 x, q11l, q01h;\n\t"                                              \
  "addc.u32 y, q11h, 0;\n\t"                                                    \
  "add.cc.u32 x, x, q10h;\n\t"                                                  \
  "addc.u32 y, y, 0;\n\t"

__device__ __forceinline__ uint64_t mont_mul_e(uint64_t a, uint64_t b, uint64_t n, uint64_t ninv) {
  IP_MONT_C_DECL
  asm("{\n\t" IP_MONT_C_REGS
      "mul.wide.u32 w, %2, %4;\n\t"
      "mov.b64 {p00l, p00h}, w;\n\t"
      "mul.wide.u32 w, %2, %5;\n\t"
      "mov.b64 {p01l, p01h}, w;\n\t"
      "mul.wide.u32 w, %3, %4;\n\t"
      "mov.b64 {p10l, p10h}, w;\n\t"
      IP_MONT_E_TAIL(IP_MONT_E_BODY) "}" IP_MONT_C_OPERANDS);
  return ((uint64_t)r1 << 32) | r0;
}

__device__ __forceinline__ uint64_t mont_sqr_e(uint64_t a, uint64_t n, uint64_t ninv) {
  const uint64_t b = a;
  IP_MONT_C_DECL
  asm("{\n\t" IP_MONT_C_REGS
      "mul.wide.u32 w, %2, %4;\n\t"
      "mov.b64 {p00l, p00h}, w;\n\t"
      "mul.wide.u32 w, %2, %5;\n\t"
      "mov.b64 {p01l, p01h}, w;\n\t"
      "mov.u32 p10l, p01l;\n\t"
      "mov.u32 p10h, p01h;\n\t"
      IP_MONT_E_TAIL(IP_MONT_E_BODY) "}" IP_MONT_C_OPERANDS);
  return ((uint64_t)r1 << 32) | r0;
}
#undef IP_MONT_E_TAIL
#undef IP_MONT_E_BODY
#undef IP_MONT_C_DECL
#undef IP_MONT_C_REGS
#undef IP_MONT_C_TAIL
#undef IP_MONT_C_OPERANDS

// Formulations 7 and 8: the same product and reduction, with the partial sums
// folded into the wide products through their 64-bit addend (mad.wide.u32),
// since every such sum stays below 2^64:
//   U  = a0 b1 + hi(a0 b0)            V  = a1 b0 + lo(U)
//   T  = a1 b1 + hi(U) + hi(V)        a b = T 2^64 + lo(V) 2^32 + lo(a0 b0)
//   V2 = m1 n0 + lo(m0 n1)            W2 = m1 n1 + hi(m0 n1) + hi(V2)
//   hi64(m n) = W2 + c, c = [lo(V2) > bits 32..63 of a b] (m0 n0 is not formed)
//   r = T - W2 - c, plus n when negative.
// Squaring (formulation 7): U = c + hi(a0^2), V = c + lo(U) with c = a0 a1
// formed once; formulation 8 squares with the multiplication.
#define IP_MONT_D_REDUCE                                                        \
  /* m = (t1:t0) n^-1 mod 2^64 */                                               \
  "mul.wide.u32 w, t0, %8;\n\t"                                                \
  "mov.b64 {m0, m1}, w;\n\t"                                                   \
  "mad.lo.u32 m1, t0, %9, m1;\n\t"                                             \
  "mad.lo.u32 m1, t1, %8, m1;\n\t"                                             \
  /* V2 = m1 n0 + lo(m0 n1); W2 = m1 n1 + hi(m0 n1) + hi(V2) */                 \
  "mul.wide.u32 w, m0, %7;\n\t"                                                \
  "mov.b64 {ql, qh}, w;\n\t"                                                   \
  "cvt.u64.u32 v2, ql;\n\t"                                                    \
  "mad.wide.u32 v2, m1, %6, v2;\n\t"                                           \
  "mov.b64 {v2l, v2h}, v2;\n\t"                                                \
  "add.cc.u32 sl, qh, v2h;\n\t"                                                \
  "addc.u32 sh, 0, 0;\n\t"                                                     \
  "mov.b64 w, {sl, sh};\n\t"                                                   \
  "mad.wide.u32 w, m1, %7, w;\n\t"                                             \
  "mov.b64 {x, y}, w;\n\t"                                                     \
  /* r = T - W2 - c, c the borrow of t1 - lo(V2); + n if negative */            \
  "mov.b64 {t2, t3}, tt;\n\t"                                                  \
  "sub.cc.u32 bo, t1, v2l;\n\t"                                                \
  "subc.cc.u32 %0, t2, x;\n\t"                                                 \
  "subc.cc.u32 %1, t3, y;\n\t"                                                 \
  "subc.u32 bo, 0, 0;\n\t"                                                     \
  "and.b32 x, bo, %6;\n\t"                                                     \
  "and.b32 y, bo, %7;\n\t"                                                     \
  "add.cc.u32 %0, %0, x;\n\t"                                                  \
  "addc.u32 %1, %1, y;\n\t"
#define IP_MONT_D_REGS                                                          \
  ".reg .u32 t0, t1, t2, t3, h, ul, uh, vh, m0, m1, ql, qh, v2l, v2h;\n\t"      \
  ".reg .u32 sl, sh, x, y, bo;\n\t"                                            \
  ".reg .u64 w, u, v, v2, tt;\n\t"

// Operands as formulation 6: %0 %1 result words; %2 %3 a; %4 %5 b; %6 %7 n;
// %8 %9 n^-1.
__device__ __forceinline__ uint64_t mont_mul_d(uint64_t a, uint64_t b, uint64_t n, uint64_t ninv) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  const uint32_t i0 = (uint32_t)ninv, i1 = (uint32_t)(ninv >> 32);
  uint32_t r0, r1;
  asm("{\n\t" IP_MONT_D_REGS
      "mul.wide.u32 w, %2, %4;\n\t"
      "mov.b64 {t0, h}, w;\n\t"
      "cvt.u64.u32 u, h;\n\t"
      "mad.wide.u32 u, %2, %5, u;\n\t"          // U = a0 b1 + hi(a0 b0)
      "mov.b64 {ul, uh}, u;\n\t"
      "cvt.u64.u32 v, ul;\n\t"
      "mad.wide.u32 v, %3, %4, v;\n\t"          // V = a1 b0 + lo(U)
      "mov.b64 {t1, vh}, v;\n\t"
      "add.cc.u32 sl, uh, vh;\n\t"
      "addc.u32 sh, 0, 0;\n\t"
      "mov.b64 tt, {sl, sh};\n\t"
      "mad.wide.u32 tt, %3, %5, tt;\n\t"        // T = a1 b1 + hi(U) + hi(V)
      IP_MONT_D_REDUCE "}"
      : "=r"(r0), "=r"(r1)
      : "r"(a0), "r"(a1), "r"(b0), "r"(b1), "r"(n0), "r"(n1), "r"(i0), "r"(i1));
  return ((uint64_t)r1 << 32) | r0;
}

__device__ __forceinline__ uint64_t mont_sqr_d(uint64_t a, uint64_t n, uint64_t ninv) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  const uint32_t i0 = (uint32_t)ninv, i1 = (uint32_t)(ninv >> 32);
  uint32_t r0, r1;
  asm("{\n\t" IP_MONT_D_REGS
      ".reg .u32 cl, ch;\n\t"
      "mul.wide.u32 w, %2, %2;\n\t"
      "mov.b64 {t0, h}, w;\n\t"
      "mul.wide.u32 w, %2, %3;\n\t"             // c = a0 a1
      "mov.b64 {cl, ch}, w;\n\t"
      "add.cc.u32 ul, cl, h;\n\t"               // U = c + hi(a0^2)
      "addc.u32 uh, ch, 0;\n\t"
      "add.cc.u32 t1, cl, ul;\n\t"              // V = c + lo(U)
      "addc.u32 vh, ch, 0;\n\t"
      "add.cc.u32 sl, uh, vh;\n\t"
      "addc.u32 sh, 0, 0;\n\t"
      "mov.b64 tt, {sl, sh};\n\t"
      "mad.wide.u32 tt, %3, %3, tt;\n\t"        // T = a1^2 + hi(U) + hi(V)
      IP_MONT_D_REDUCE "}"
      : "=r"(r0), "=r"(r1)
      : "r"(a0), "r"(a1), "r"(a0), "r"(a1), "r"(n0), "r"(n1), "r"(i0), "r"(i1));
  return ((uint64_t)r1 << 32) | r0;
}
#undef IP_MONT_D_REDUCE
#undef IP_MONT_D_REGS
#endif

// Word-level Montgomery multiplication (Montgomery 1985, two 32-bit words
// of reduction per 64-bit product), written with 32x32+64 -> 64 wide
// multiply-adds so that every partial product and its carry-in take one
// IMAD.WIDE.  q = -n^-1 mod 2^32.  Inputs a, b < n; result in [0, n).
//   product:   4 wide  (a0b0, a0b1, a1b0, a1b1)
//   reduction: 2 x (m = t_i q mod 2^32, then m n0 and m n1 wide)
// The running value after the product is t3:t2:t1:t0 < n^2; adding
// m n + m' n 2^32 keeps it below 2n 2^64, so one extra bit (t4) suffices.
IP_HD uint64_t mont_reduce_w(uint32_t t0, uint32_t t1, uint64_t H, uint64_t n, uint32_t q) {
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  // step 1: cancel t0
  uint32_t m = t0 * q;
  uint64_t acc = (uint64_t)m * n0 + t0;
  acc = (uint64_t)m * n1 + t1 + (acc >> 32);
  t1 = (uint32_t)acc;
  const uint64_t c = acc >> 32;
  H += c;
  uint32_t t4 = H < c;
  // step 2: cancel t1
  m = t1 * q;
  acc = (uint64_t)m * n0 + t1;
  acc = (uint64_t)m * n1 + (uint32_t)H + (acc >> 32);
  const uint64_t U = (H >> 32) + (acc >> 32) + ((uint64_t)t4 << 32);  // < 2^33
  uint64_t r = (U << 32) | (uint32_t)acc;
  return ((U >> 32) != 0 || r >= n) ? r - n : r;
}

IP_HD uint64_t mont_mul_w(uint64_t a, uint64_t b, uint64_t n, uint32_t q) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
  uint64_t acc = (uint64_t)a0 * b0;
  const uint32_t t0 = (uint32_t)acc;
  acc = (uint64_t)a0 * b1 + (acc >> 32);
  const uint64_t c1 = acc >> 32;
  acc = (uint64_t)a1 * b0 + (uint32_t)acc;
  const uint32_t t1 = (uint32_t)acc;
  const uint64_t H = (uint64_t)a1 * b1 + c1 + (acc >> 32);  // top 64 bits of a*b
  return mont_reduce_w(t0, t1, H, n, q);
}

// a^2: a0^2 + 2 a0 a1 2^32 + a1^2 2^64 with three wide products.
IP_HD uint64_t mont_sqr_w(uint64_t a, uint64_t n, uint32_t q) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint64_t L = (uint64_t)a0 * a0;
  const uint64_t X = (uint64_t)a0 * a1;
  const uint64_t D = X << 1;                   // low 64 bits of 2X
  const uint64_t dt = X >> 63;                 // bit 64 of 2X
  const uint64_t u = (L >> 32) + (uint32_t)D;  // < 2^33
  const uint32_t t0 = (uint32_t)L, t1 = (uint32_t)u;
  // top 64 bits of a^2 (cannot overflow: a^2 < 2^128)
  const uint64_t H = (uint64_t)a1 * a1 + (D >> 32) + (u >> 32) + (dt << 32);
  return mont_reduce_w(t0, t1, H, n, q);
}

// Fused product-scanning Montgomery multiplication (q = -n^-1 mod 2^32).
// The product a*b and the two word-level reduction steps are interleaved so
// that every carry enters as the 64-bit addend of a 32x32+64 -> 64 wide
// multiply-add, which costs nothing extra:
//   acc0 = m0 n0 + t0         (m0 = t0 q, so the low word of acc0 is 0)
//   X = a0 b1 + hi(a0 b0),  Y = a1 b0 + lo(X),  Z = m0 n1 + lo(Y)
//   w1 + k1 2^32 = lo(Z) + hi(acc0)                (word 1 of a b + m0 n)
//   V = m1 n0 + w1            (m1 = w1 q, so the low word of V is 0)
//   (a b + m0 n + m1 n 2^32) / 2^64
//       = (a1 b1 + hi(X)) + (m1 n1 + hi(Y)) + hi(Z) + hi(V) + k1  < 2n.
// Eight wide products and two 32-bit products; the result is reduced to
// [0, n) by one conditional subtraction.
IP_HD uint64_t mont_fused_tail(uint64_t U, uint64_t U2, uint32_t hz, uint32_t hv, uint32_t k1,
                               uint64_t n) {
  const uint64_t small = (uint64_t)hz + hv + k1;  // < 2^33
  uint64_t r = U + U2;
  uint32_t c = r < U;
  r += small;
  c += r < small;
  return (c || r >= n) ? r - n : r;
}

IP_HD uint64_t mont_mul_f(uint64_t a, uint64_t b, uint64_t n, uint32_t q) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  const uint64_t P = (uint64_t)a0 * b0;
  const uint32_t t0 = (uint32_t)P;
  const uint32_t m0 = t0 * q;
  const uint64_t acc0 = (uint64_t)m0 * n0 + t0;
  const uint64_t X = (uint64_t)a0 * b1 + (P >> 32);
  const uint64_t Y = (uint64_t)a1 * b0 + (uint32_t)X;
  const uint64_t Z = (uint64_t)m0 * n1 + (uint32_t)Y;
  const uint64_t W1 = (Z & 0xFFFFFFFFull) + (acc0 >> 32);  // < 2^33
  const uint32_t w1 = (uint32_t)W1;
  const uint32_t m1 = w1 * q;
  const uint64_t V = (uint64_t)m1 * n0 + w1;
  const uint64_t U = (uint64_t)a1 * b1 + (X >> 32);
  const uint64_t U2 = (uint64_t)m1 * n1 + (Y >> 32);
  return mont_fused_tail(U, U2, (uint32_t)(Z >> 32), (uint32_t)(V >> 32), (uint32_t)(W1 >> 32), n);
}

// Squaring in the fused form: the cross product a0 a1 is computed once and
// used for both X and Y (one wide product fewer, two 64-bit adds more).
IP_HD uint64_t mont_sqr_f(uint64_t a, uint64_t n, uint32_t q) {
  const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  const uint64_t P = (uint64_t)a0 * a0;
  const uint32_t t0 = (uint32_t)P;
  const uint32_t m0 = t0 * q;
  const uint64_t acc0 = (uint64_t)m0 * n0 + t0;
  const uint64_t C = (uint64_t)a0 * a1;
  const uint64_t X = C + (P >> 32);          // cannot overflow: C <= (2^32-1)^2
  const uint64_t Y = C + (uint32_t)X;
  const uint64_t Z = (uint64_t)m0 * n1 + (uint32_t)Y;
  const uint64_t W1 = (Z & 0xFFFFFFFFull) + (acc0 >> 32);
  const uint32_t w1 = (uint32_t)W1;
  const uint32_t m1 = w1 * q;
  const uint64_t V = (uint64_t)m1 * n0 + w1;
  const uint64_t U = (uint64_t)a1 * a1 + (X >> 32);
  const uint64_t U2 = (uint64_t)m1 * n1 + (Y >> 32);
  return mont_fused_tail(U, U2, (uint32_t)(Z >> 32), (uint32_t)(V >> 32), (uint32_t)(W1 >> 32), n);
}

// 2x mod n for x < n (ModAdd of x to itself, Sec. 2.2): if 2x overflows 64
// bits it is certainly >= n, and the wrapped difference is exact.
IP_HD uint64_t mod_dbl(uint64_t x, uint64_t n) {
  uint64_t y = x << 1;
  return ((int64_t)x < 0 || y >= n) ? y - n : y;
}

// 2^64 mod n for odd n > 1 without a division: with k the bit length of n,
// 2^(k-1) < n < 2^k, so 2^k mod n = 2^k - n; then 64 - k modular doublings.
IP_HD uint64_t pow2_64_mod(uint64_t n) {
  const int k = 64 - clz64(n);
  uint64_t x = (k == 64) ? (0 - n) : ((1ull << k) - n);
  for (int i = k; i < 64; ++i) x = mod_dbl(x, n);
  return x;
}

IP_HD Mont64 mont64_setup(uint64_t n) {
  Mont64 m;
  m.n = n;
  const uint32_t i32 = inv32((uint32_t)n);
  uint64_t i64 = i32;
  i64 *= 2 - n * i64;  // one Newton step lifts the 32-bit inverse to 64 bits
  m.ninv = i64;
  m.q = 0u - i32;
  m.one = pow2_64_mod(n);  // R mod n
  m.mone = n - m.one;
  return m;
}

// The Montgomery multiplication and squaring used by the kernels, selected
// at compile time (the tuning parameter mont_impl picks the instantiation):
//   0: 128-bit product, REDC hi(ab) - hi(mn); squaring with one cross product
//   1: word-level REDC with wide multiply-adds (mont_mul_w / mont_sqr_w)
//   2: 128-bit product with a word-level REDC in PTX carry chains (device)
//   3: fused product-scanning multiplication and squaring (mont_mul_f/_sqr_f)
//   4: 128-bit multiplication with the fused squaring
//   5: 128-bit multiplication, squaring as a general multiplication
//   6: 128-bit form in 32-bit words as PTX, no m0 n0 product (device)
//   7: formulation 6 with the partial sums in the wide products' addends
//   8: formulation 7, squaring as a general multiplication
//   9: formulation 6 with the final correction on the multiply pipe
template <int kImpl>
struct MontOps;

template <>
struct MontOps<0> {
  static IP_HD uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) { return mont_mul(a, b, M.n, M.ninv); }
  static IP_HD uint64_t sqr(uint64_t a, const Mont64& M) { return mont_sqr_h(a, M.n, M.ninv); }
};

template <>
struct MontOps<1> {
  static IP_HD uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) { return mont_mul_w(a, b, M.n, M.q); }
  static IP_HD uint64_t sqr(uint64_t a, const Mont64& M) { return mont_sqr_w(a, M.n, M.q); }
};

template <>
struct MontOps<3> {
  static IP_HD uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) { return mont_mul_f(a, b, M.n, M.q); }
  static IP_HD uint64_t sqr(uint64_t a, const Mont64& M) { return mont_sqr_f(a, M.n, M.q); }
};

// 4: the 128-bit-form multiplication with the fused squaring
template <>
struct MontOps<4> {
  static IP_HD uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) { return mont_mul(a, b, M.n, M.ninv); }
  static IP_HD uint64_t sqr(uint64_t a, const Mont64& M) { return mont_sqr_f(a, M.n, M.q); }
};

// 5: the 128-bit multiplication, squaring as a general multiplication
template <>
struct MontOps<5> {
  static IP_HD uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) { return mont_mul(a, b, M.n, M.ninv); }
  static IP_HD uint64_t sqr(uint64_t a, const Mont64& M) { return mont_mul(a, a, M.n, M.ninv); }
};

#if defined(__CUDACC__)
// 6: the word-level PTX form of the 128-bit REDC (mont_mul_c / mont_sqr_c)
template <>
struct MontOps<6> {
  static __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) {
    return mont_mul_c(a, b, M.n, M.ninv);
  }
  static __device__ __forceinline__ uint64_t sqr(uint64_t a, const Mont64& M) {
    return mont_sqr_c(a, M.n, M.ninv);
  }
};

template <>
struct MontOps<9> {
  static __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) {
    return mont_mul_e(a, b, M.n, M.ninv);
  }
  static __device__ __forceinline__ uint64_t sqr(uint64_t a, const Mont64& M) {
    return mont_sqr_e(a, M.n, M.ninv);
  }
};

template <>
struct MontOps<7> {
  static __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) {
    return mont_mul_d(a, b, M.n, M.ninv);
  }
  static __device__ __forceinline__ uint64_t sqr(uint64_t a, const Mont64& M) {
    return mont_sqr_d(a, M.n, M.ninv);
  }
};

template <>
struct MontOps<8> {
  static __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) {
    return mont_mul_d(a, b, M.n, M.ninv);
  }
  static __device__ __forceinline__ uint64_t sqr(uint64_t a, const Mont64& M) {
    return mont_mul_d(a, a, M.n, M.ninv);
  }
};

// Formulations 16 and 17: formulation 6 with every operation counted, for
// the measurement entry point isprime_count_ops (16 in the base-2 kernel, 17
// in the six-base kernel).  Per operation the warp's first active lane adds
// one warp-level issue and the number of active lanes to a counter of this
// translation unit (64 copies, picked by block, to spread the atomics).
// Kinds: 0 squaring, 1 product, 2 multiplication by 2^w (base-2 window step).
constexpr int kOpKinds = 3;
constexpr int kOpSpread = 64;
static __device__ unsigned long long g_ip_ops[2][kOpKinds][2][kOpSpread];

template <int kImpl>
__device__ __forceinline__ void op_note(int kind) {
  if constexpr (kImpl == 16 || kImpl == 17) {
    const unsigned m = __activemask();
    if ((int)(threadIdx.x & 31) == __ffs(m) - 1) {
      unsigned long long* c = g_ip_ops[kImpl - 16][kind][0];
      atomicAdd(&c[blockIdx.x % kOpSpread], 1ull);
      atomicAdd(&c[kOpSpread + blockIdx.x % kOpSpread], (unsigned long long)__popc(m));
    }
  }
}

template <>
struct MontOps<16> {
  static __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) {
    op_note<16>(1);
    return mont_mul_c(a, b, M.n, M.ninv);
  }
  static __device__ __forceinline__ uint64_t sqr(uint64_t a, const Mont64& M) {
    op_note<16>(0);
    return mont_sqr_c(a, M.n, M.ninv);
  }
};

template <>
struct MontOps<17> {
  static __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) {
    op_note<17>(1);
    return mont_mul_c(a, b, M.n, M.ninv);
  }
  static __device__ __forceinline__ uint64_t sqr(uint64_t a, const Mont64& M) {
    op_note<17>(0);
    return mont_sqr_c(a, M.n, M.ninv);
  }
};

template <>
struct MontOps<2> {
  static __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b, const Mont64& M) {
    return mont_mul_p(a, b, M.n, M.q);
  }
  static __device__ __forceinline__ uint64_t sqr(uint64_t a, const Mont64& M) {
    return mont_mul_p(a, a, M.n, M.q);
  }
};
#endif

// R^2 mod n from R mod n: 8 doublings give R 2^8; each Montgomery squaring
// maps R 2^k to R 2^(2k): 2^8 -> 2^16 -> 2^32 -> 2^64.
template <int kImpl = 0>
IP_HD uint64_t mont64_r2(const Mont64& M) {
  uint64_t x = M.one;
  IP_UNROLL
  for (int i = 0; i < 8; ++i) x = mod_dbl(x, M.n);
  x = MontOps<kImpl>::sqr(x, M);
  x = MontOps<kImpl>::sqr(x, M);
  x = MontOps<kImpl>::sqr(x, M);
  return x;
}

// Strong probable-prime test to base 2 (Sec. 2.1), n odd, n > 2.
// 2^d by left-to-right binary exponentiation where "multiply by the base"
// is a modular doubling.  The exponent is processed from the top in whole
// nibbles (leading zero bits square the Montgomery 1, which stays 1), with a
// 4-way unrolled body and the exponent bit read from a shifting register.
template <int kImpl = 0>
IP_HD bool sprp2_64(const Mont64& M, uint64_t d, int s) {
  const uint64_t n = M.n;
  const int nib = (64 - clz64(d) + 3) >> 2;  // nibbles in d (d >= 1)
  uint64_t e = d << (64 - 4 * nib);          // exponent bits left-aligned
  uint64_t x = M.one;
  for (int k = 0; k < nib; ++k) {
    IP_UNROLL
    for (int j = 0; j < 4; ++j) {
      x = MontOps<kImpl>::sqr(x, M);
      const uint64_t y = mod_dbl(x, n);
      x = ((int64_t)e < 0) ? y : x;
      e <<= 1;
    }
  }
  if (x == M.one || x == M.mone) return true;
  for (int r = 1; r < s; ++r) {
    x = MontOps<kImpl>::sqr(x, M);
    if (x == M.mone) return true;
    if (x == M.one) return false;
  }
  return false;
}

// A 32-bit residue of n = n1 2^32 + n0 modulo an odd m < 2^32 (mneg =
// -m^-1 mod 2^32), by one Montgomery reduction step:
//   q = n0 mneg mod 2^32,  u = q m + n0 < 2^64 (its low word is 0),
//   t = n1 + u / 2^32 = (n + q m) / 2^32,
// so t = n 2^-32 (mod m) and t <= 2^32 - 1 + m (u / 2^32 <= m); subtracting m
// once when t >= m leaves r < 2^32 with the same residue.  2^-32 is a unit
// modulo every odd p | m, so p | n exactly when p | r, and p | r is the
// 32-bit test r p^-1 mod 2^32 <= floor((2^32 - 1) / p).
IP_HD uint32_t mont_residue32(uint32_t n0, uint32_t n1, uint32_t m, uint32_t mneg) {
  const uint32_t q = n0 * mneg;
  const uint64_t u = (uint64_t)q * m + n0;
  const uint64_t t = (uint64_t)n1 + (u >> 32);
  return (uint32_t)(t >= m ? t - m : t);
}

// Second trial-division stage: true when a prime of the first kGroups groups
// of T divides n (n > 457, so such a divisor makes n composite): one residue
// per group of three primes, each prime tested on it.
template <int kGroups>
IP_HD bool td2_divisible(uint64_t n, const Td2Table& T) {
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  bool div = false;
  IP_UNROLL
  for (int g = 0; g < kGroups; ++g) {
    const uint32_t r = mont_residue32(n0, n1, T.m[g], T.mneg[g]);
    IP_UNROLL
    for (int k = 3 * g; k < 3 * g + 3; ++k) div |= (uint32_t)(r * T.inv[k]) <= T.lim[k];
  }
  return div;
}

// Trial division of a 64-bit n by the odd primes 3..53 on two residues (the
// groups A and B of tables.cuh): true when one of them divides n.  inv and lim
// are the primes' 32-bit inverses and limits in the order of kTdPrimeList.
IP_HD bool td_pair_divisible(uint64_t n, const uint32_t* inv, const uint32_t* lim) {
  const uint32_t n0 = (uint32_t)n, n1 = (uint32_t)(n >> 32);
  const uint32_t ra = mont_residue32(n0, n1, kTdPairA, kTdPairNegA);
  const uint32_t rb = mont_residue32(n0, n1, kTdPairB, kTdPairNegB);
  bool div = false;
  IP_UNROLL
  for (int i = 0; i < kFoldPrimes; ++i)
    div |= (uint32_t)((td_pair_in_a(i) ? ra : rb) * inv[i]) <= lim[i];
  return div;
}

// Finishes a strong test once x = a^d (Montgomery form) is known.
template <int kImpl = 0>
IP_HD bool sprp_tail64(const Mont64& M, uint64_t x, int s) {
  if (x == M.one || x == M.mone) return true;
  for (int r = 1; r < s; ++r) {
    x = MontOps<kImpl>::sqr(x, M);
    if (x == M.mone) return true;
    if (x == M.one) return false;
  }
  return false;
}

// a^d for a base a < n given in Montgomery form (aR), plain left-to-right
// binary exponentiation (host reference for the windowed device kernels).
template <int kImpl = 0>
IP_HD uint64_t mont_pow_binary(const Mont64& M, uint64_t aR, uint64_t d) {
  uint64_t x = M.one;
  for (int b = 63 - clz64(d); b >= 0; --b) {
    x = MontOps<kImpl>::sqr(x, M);
    if ((d >> b) & 1) x = MontOps<kImpl>::mul(x, aR, M);
  }
  return x;
}

// ---------------------------------------------------------------------------
// Strong Lucas probable-prime test with Selfridge's parameters (Baillie and
// Wagstaff, Math. Comp. 35, 1980): D is the first of 5, -7, 9, -11, ... with
// Jacobi symbol (D/n) = -1, P = 1, Q = (1 - D)/4; with n + 1 = 2^s d, d odd,
// n passes if U_d = 0 or V_(d 2^r) = 0 (mod n) for some 0 <= r < s.  After
// the base-2 strong test this is the Baillie-PSW test.
// ---------------------------------------------------------------------------

// Jacobi symbol (a/n) for odd n > 0 and |a| < 2^62, binary algorithm.
IP_HD int jacobi_symbol(int64_t a, uint64_t n) {
  uint64_t x = a >= 0 ? (uint64_t)a % n : (n - ((uint64_t)(-a) % n)) % n;
  uint64_t m = n;
  int t = 1;
  while (x != 0) {
    while ((x & 1) == 0) {
      x >>= 1;
      const uint64_t r = m & 7;
      if (r == 3 || r == 5) t = -t;
    }
    const uint64_t tmp = x;
    x = m;
    m = tmp;
    if ((x & 3) == 3 && (m & 3) == 3) t = -t;
    x %= m;
  }
  return m == 1 ? t : 0;
}

// Jacobi symbol (D/n) for odd n > 0 and a small odd D (|D| < 2^16): by
// reciprocity (D/n) = sign * (n mod |D| / |D|), and n mod |D| splits into
// 32-bit steps (n = h 2^32 + l), so everything after that is 32-bit.
IP_HD int jacobi_small(int32_t D, uint64_t n) {
  int t = 1;
  uint32_t a = (uint32_t)(D < 0 ? -D : D);
  if (D < 0 && (n & 3) == 3) t = -t;  // (-1/n) = (-1)^((n-1)/2)
  if ((a & 3) == 3 && (n & 3) == 3) t = -t;  // reciprocity for odd a, n
  const uint32_t h = (uint32_t)(n >> 32), l = (uint32_t)n;
  const uint32_t c = (0xFFFFFFFFu % a + 1u) % a;  // 2^32 mod a
  uint32_t x = ((h % a) * c % a + l % a) % a;     // n mod a; (h % a) * c < a^2 < 2^32
  uint32_t m = a;
  while (x != 0) {
    while ((x & 1) == 0) {
      x >>= 1;
      const uint32_t r = m & 7;
      if (r == 3 || r == 5) t = -t;
    }
    const uint32_t tmp = x;
    x = m;
    m = tmp;
    if ((x & 3) == 3 && (m & 3) == 3) t = -t;
    x %= m;
  }
  return m == 1 ? t : 0;
}

// floor(sqrt(n))^2 == n for n < 2^64.
IP_HD bool is_square64(uint64_t n) {
  uint64_t r = (uint64_t)sqrt((double)n);
  if (r > 0xFFFFFFFFull) r = 0xFFFFFFFFull;
  while (r * r > n) --r;
  while (r < 0xFFFFFFFFull && (r + 1) * (r + 1) <= n) ++r;
  return r * r == n;
}

IP_HD uint64_t mod_add(uint64_t a, uint64_t b, uint64_t n) {  // a, b < n
  const uint64_t s = a + b;
  return (s < a || s >= n) ? s - n : s;
}
IP_HD uint64_t mod_sub(uint64_t a, uint64_t b, uint64_t n) {  // a, b < n
  return a >= b ? a - b : a - b + n;
}
IP_HD uint64_t mod_half(uint64_t x, uint64_t n) {  // x / 2 mod n for odd n, x < n
  return (x & 1) ? (x >> 1) + (n >> 1) + 1 : x >> 1;
}

// Montgomery form of a small signed integer c (|c| < n).
template <int kImpl>
IP_HD uint64_t mont_from_small(int64_t c, uint64_t r2, const Mont64& M) {
  const uint64_t m = MontOps<kImpl>::mul(c >= 0 ? (uint64_t)c : (uint64_t)(-c), r2, M);
  return (c >= 0 || m == 0) ? m : M.n - m;
}

// Selfridge's D for odd n: the first of 5, -7, 9, -11, ... with (D/n) = -1.
// Returns 0 with *D set, or 1 if the search shows n composite (a D sharing a
// factor with n, or n a perfect square, for which no such D exists).
IP_HD int lucas_next_D(uint64_t n, int32_t* D, int* k) {  // one search step: -1 still searching
  const int j = jacobi_small(*D, n);
  if (j == -1) return 0;
  if (j == 0) return 1;                          // gcd(D, n) > 1 and |D| < n
  if (*k == 8 && is_square64(n)) return 1;       // squares have no D with (D/n) = -1
  *D = *D > 0 ? -(*D + 2) : -*D + 2;
  ++*k;
  return -1;
}

// The Lucas ladder for U_d, V_d (P = 1, Q = (1 - D)/4) over the low `nbits`
// bits of d (nbits >= bitlen(d)), then the strong condition.  It starts from
// k = 0: (U_0, V_0, Q^0) = (0, 2, 1) is fixed by doubling, so leading zero
// bits cost time but not correctness; a warp can run one uniform count.
template <int kImpl>
IP_HD bool lucas_ladder(uint64_t n, int32_t D, int nbits) {
  using Ops = MontOps<kImpl>;
  const int64_t Q = (1 - (int64_t)D) / 4;
  const Mont64 M = mont64_setup(n);
  const uint64_t r2 = mont64_r2<kImpl>(M);
  const uint64_t Dm = mont_from_small<kImpl>(D, r2, M);
  const uint64_t Qm = mont_from_small<kImpl>(Q, r2, M);
  uint64_t d = n + 1;
  const int s = ctz64(d);
  d >>= s;
  uint64_t U = 0, V = mod_dbl(M.one, n), Qk = M.one;
  for (int b = nbits - 1; b >= 0; --b) {
    // k -> 2k
    U = Ops::mul(U, V, M);
    V = mod_sub(Ops::sqr(V, M), mod_dbl(Qk, n), n);
    Qk = Ops::sqr(Qk, M);
    // 2k -> 2k + 1 when the bit is set (computed always and selected)
    const uint64_t U1 = mod_half(mod_add(U, V, n), n);
    const uint64_t V1 = mod_half(mod_add(Ops::mul(Dm, U, M), V, n), n);
    const uint64_t Q1 = Ops::mul(Qk, Qm, M);
    const bool bit = (d >> b) & 1;
    U = bit ? U1 : U;
    V = bit ? V1 : V;
    Qk = bit ? Q1 : Qk;
  }
  if (U == 0 || V == 0) return true;
  for (int r = 1; r < s; ++r) {
    V = mod_sub(Ops::sqr(V, M), mod_dbl(Qk, n), n);
    if (V == 0) return true;
    Qk = Ops::sqr(Qk, M);
  }
  return false;
}

IP_HD int lucas_bits(uint64_t n) {  // bit length of the odd part of n + 1
  uint64_t d = n + 1;
  d >>= ctz64(d);
  return 64 - clz64(d);
}

// n odd, n > 2^32, not divisible by small primes.  Returns the strong
// Lucas probable-prime verdict (single-lane form).
template <int kImpl>
IP_HD bool strong_lucas_selfridge(uint64_t n) {
  if (n == ~0ull) return false;  // 2^64 - 1 = 3 * 5 * 17 * 257 * 641 * 65537 * 6700417
  int32_t D = 5;
  int k = 0, st;
  while ((st = lucas_next_D(n, &D, &k)) < 0) {
  }
  if (st) return false;
  return lucas_ladder<kImpl>(n, D, lucas_bits(n));
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

// 2^32 mod n for odd n > 1, as pow2_64_mod: 2^k - n, then 32 - k doublings.
IP_HD uint32_t pow2_32_mod(uint32_t n) {
  const int k = 32 - clz32(n);
  uint32_t x = (k == 32) ? (0u - n) : ((1u << k) - n);
  for (int i = k; i < 32; ++i) x = mod_dbl32(x, n);
  return x;
}

IP_HD Mont32 mont32_setup(uint32_t n) {
  Mont32 m;
  m.n = n;
  m.ninv = inv32(n);
  m.one = pow2_32_mod(n);
  m.mone = n - m.one;
  return m;
}

// R^2 mod n (R = 2^32) from R mod n: 8 doublings give R 2^8, two Montgomery
// squarings map it to R 2^16 and R 2^32 = R^2.
IP_HD uint32_t mont32_r2(const Mont32& M) {
  uint32_t x = M.one;
  for (int i = 0; i < 8; ++i) x = mod_dbl32(x, M.n);
  x = mont_mul32(x, x, M.n, M.ninv);
  return mont_mul32(x, x, M.n, M.ninv);
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
    const uint32_t aR = mont_mul32(a, mont32_r2(M), n, ninv);  // a R mod n
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
