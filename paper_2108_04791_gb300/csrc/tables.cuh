// tables.cuh -- compile-time constants for the primality kernels.
//
// Trial division by small primes (removing multiples of small primes before
// the expensive test, Sec. 6.1.2, and keeping divisions few, Sec. 6.1.3) is
// done without any division: for odd p and any n < 2^64,
//     p | n  <=>  n * p^-1 mod 2^64 <= floor((2^64 - 1) / p)
// (Granlund and Montgomery, PLDI 1994, Sec. 9).  The inverses and limits are
// generated at compile time by constexpr Newton iterations.
#pragma once
#include <stdint.h>

namespace ip {

// The Miller-Rabin bases of Eq. 4 (exact for all n < 2^64), and the three
// bases that are exact below 4,759,123,141 > 2^32 (Jaeschke 1993).
constexpr int kNumBases64 = 7;
constexpr uint32_t kBases64[kNumBases64] = {2u,      325u,     9375u,      28178u,
                                            450775u, 9780504u, 1795265022u};
constexpr int kNumBases32 = 3;
constexpr uint32_t kBases32[kNumBases32] = {2u, 7u, 61u};

struct BaseTable {
  uint32_t b64[kNumBases64];
  uint32_t b32[kNumBases32];
};

constexpr BaseTable make_base_table() {
  BaseTable t{};
  for (int i = 0; i < kNumBases64; ++i) t.b64[i] = kBases64[i];
  for (int i = 0; i < kNumBases32; ++i) t.b32[i] = kBases32[i];
  return t;
}

// Odd primes 3..251 available for trial division.
constexpr int kMaxTdPrimes = 53;
constexpr uint32_t kTdPrimeList[kMaxTdPrimes] = {
    3,   5,   7,   11,  13,  17,  19,  23,  29,  31,  37,  41,  43,  47,
    53,  59,  61,  67,  71,  73,  79,  83,  89,  97,  101, 103, 107, 109,
    113, 127, 131, 137, 139, 149, 151, 157, 163, 167, 173, 179, 181, 191,
    193, 197, 199, 211, 223, 227, 229, 233, 239, 241, 251};
// The prime after 251; (next prime after the last tested)^2 bounds the range
// where surviving trial division already proves primality.
constexpr uint32_t kTdNextPrimeAfterList = 257;

struct TdTable {
  uint64_t inv64[kMaxTdPrimes];
  uint64_t lim64[kMaxTdPrimes];
  uint32_t inv32[kMaxTdPrimes];
  uint32_t lim32[kMaxTdPrimes];
  uint32_t p[kMaxTdPrimes];
};

constexpr uint64_t ce_inv64(uint64_t n) {
  uint64_t x = (3 * n) ^ 2;
  for (int i = 0; i < 4; ++i) x *= 2 - n * x;
  return x;
}

constexpr TdTable make_td_table() {
  TdTable t{};
  for (int i = 0; i < kMaxTdPrimes; ++i) {
    uint64_t p = kTdPrimeList[i];
    t.p[i] = (uint32_t)p;
    t.inv64[i] = ce_inv64(p);
    t.lim64[i] = ~0ULL / p;
    t.inv32[i] = (uint32_t)ce_inv64(p);
    t.lim32[i] = 0xFFFFFFFFu / (uint32_t)p;
  }
  return t;
}

constexpr TdTable kTdHost = make_td_table();

// Folded trial division.  For k bits, 2^k = 1 (mod 2^k - 1), so the sum of
// the k-bit chunks of n is congruent to n modulo 2^k - 1, and modulo every
// prime p dividing 2^k - 1.  With k = 32, 24, 20 and 28 that sum fits in 32
// bits, so p | n is decided by the 32-bit multiply-by-inverse test on it (one
// low multiply) instead of the 64-bit one (a wide and two low multiplies):
//   2^32 - 1 = 3 * 5 * 17 * 257 * 65537
//   2^24 - 1 = 3^2 * 5 * 7 * 13 * 17 * 241
//   2^20 - 1 = 3 * 5^2 * 11 * 31 * 41
//   2^28 - 1 = 3 * 5 * 29 * 43 * 113 * 127
// fold_width(i, level) is the k whose chunk sum serves the i-th odd prime
// (0: the 64-bit test) at fold level 1 (k = 32, 24, 20) or 2 (also 28): 3, 5
// and 17 by 2^32 - 1, 7 and 13 by 2^24 - 1, 11, 31 and 41 by 2^20 - 1, 29 and
// 43 by 2^28 - 1.  It is plain arithmetic on i (no table), since device code
// calls it.  The shifts, masks and adds of the folds run on the ALU pipe, the
// tests they replace on the multiply pipe, so the level trades one pipe's
// work for the other's.
constexpr int kFoldPrimes = 15;  // 3 .. 53
constexpr int fold_width(int i, int level) {
  return level <= 0 ? 0
         : (i == 0 || i == 1 || i == 5)             ? 32
         : (i == 2 || i == 4)                       ? 24
         : (i == 3 || i == 9 || i == 11)            ? 20
         : ((i == 8 || i == 12) && level >= 2)      ? 28
                                                    : 0;
}
// Every prime given a fold divides 2^k - 1 (checked at compile time).
constexpr bool fold_widths_divide() {
  for (int level = 1; level <= 2; ++level)
    for (int i = 0; i < kMaxTdPrimes; ++i) {
      const int k = fold_width(i, level);
      if (k != 0 && (i >= kFoldPrimes || ((1ull << k) - 1) % kTdPrimeList[i] != 0)) return false;
    }
  return true;
}
static_assert(fold_widths_divide(), "a folded prime does not divide 2^k - 1");

// Trial division by two residues (td_fold 3).  The product of the odd primes
// 3..53 is below 2^64 and splits into two groups with products below 2^32:
//   A = 29 * 31 * 41 * 43 * 47 * 53 = 3,948,078,067
//   B = 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23 * 37 = 4,127,218,095
// A 64-bit n is reduced to one 32-bit residue per group (mont_residue32 in
// arith.cuh) and every prime is tested on its group's residue with the 32-bit
// multiply-by-inverse test: two reductions and fifteen 32-bit tests instead of
// chunk sums and 64-bit tests.  td_pair_in_a(i) is plain arithmetic on the
// prime's index i (no table: device code calls it).
constexpr bool td_pair_in_a(int i) { return i == 8 || i == 9 || (i >= 11 && i < kFoldPrimes); }
constexpr uint64_t td_pair_product(bool group_a) {
  uint64_t m = 1;
  for (int i = 0; i < kFoldPrimes; ++i)
    if (td_pair_in_a(i) == group_a) m *= kTdPrimeList[i];
  return m;
}
static_assert(td_pair_product(true) < ((uint64_t)1 << 32) && td_pair_product(false) < ((uint64_t)1 << 32),
              "two-residue trial division: a group's product does not fit 32 bits");
static_assert(td_pair_product(true) == 3948078067ull && td_pair_product(false) == 4127218095ull,
              "two-residue trial division: the groups");
constexpr uint32_t kTdPairA = (uint32_t)td_pair_product(true);
constexpr uint32_t kTdPairB = (uint32_t)td_pair_product(false);
constexpr uint32_t kTdPairNegA = 0u - (uint32_t)ce_inv64(kTdPairA);  // -A^-1 mod 2^32
constexpr uint32_t kTdPairNegB = 0u - (uint32_t)ce_inv64(kTdPairB);

// Second trial-division stage (tuning td2_groups): the odd primes after 53,
// tested only on the survivors of the first stage (the base-2 kernel's
// queue), where a removed value saves a whole base-2 exponentiation.  They
// come in groups of three with product m < 2^32: a 64-bit n is reduced to one
// 32-bit residue per group (td2_divisible in arith.cuh) and each prime of the
// group is tested on it with the 32-bit multiply-by-inverse test.
constexpr int kTd2MaxGroups = 24;
constexpr int kTd2Primes = 3 * kTd2MaxGroups;  // 59 .. 457

struct Td2Table {
  uint32_t m[kTd2MaxGroups];     // product of the group's three primes
  uint32_t mneg[kTd2MaxGroups];  // -m^-1 mod 2^32
  uint32_t p[kTd2Primes];
  uint32_t inv[kTd2Primes];      // p^-1 mod 2^32
  uint32_t lim[kTd2Primes];      // floor((2^32 - 1) / p)
};

constexpr bool ce_is_prime(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t d = 2; d * d <= n; ++d)
    if (n % d == 0) return false;
  return true;
}

constexpr Td2Table make_td2_table() {
  Td2Table t{};
  uint32_t c = kTdPrimeList[kFoldPrimes - 1];  // 53, the last prime of the first stage
  for (int i = 0; i < kTd2Primes; ++i) {
    c += 2;
    while (!ce_is_prime(c)) c += 2;
    t.p[i] = c;
    t.inv[i] = (uint32_t)ce_inv64(c);
    t.lim[i] = 0xFFFFFFFFu / c;
  }
  for (int g = 0; g < kTd2MaxGroups; ++g) {
    const uint64_t m = (uint64_t)t.p[3 * g] * t.p[3 * g + 1] * t.p[3 * g + 2];
    t.m[g] = (uint32_t)m;
    t.mneg[g] = 0u - (uint32_t)ce_inv64(m);
  }
  return t;
}

constexpr Td2Table kTd2Host = make_td2_table();

// Every group's product fits 32 bits and every inverse is one (compile time).
constexpr bool td2_table_ok() {
  for (int g = 0; g < kTd2MaxGroups; ++g) {
    const uint64_t m = (uint64_t)kTd2Host.p[3 * g] * kTd2Host.p[3 * g + 1] * kTd2Host.p[3 * g + 2];
    if (m >= ((uint64_t)1 << 32) || (uint32_t)(kTd2Host.m[g] * (0u - kTd2Host.mneg[g])) != 1u)
      return false;
  }
  for (int i = 0; i < kTd2Primes; ++i)
    if ((uint32_t)(kTd2Host.p[i] * kTd2Host.inv[i]) != 1u) return false;
  return kTd2Host.p[0] == 59;
}
static_assert(td2_table_ok(), "second-stage trial-division table");

}  // namespace ip
