// Host build of the device arithmetic header, for CPU unit tests only.
// Exposes the Montgomery, doubling, inverse and divisibility helpers so the
// tests can compare them with exact Python integers.
#include "../../paper_2108_04791_gb300/csrc/arith.cuh"
#include "../../paper_2108_04791_gb300/csrc/tables.cuh"

extern "C" {
uint64_t h_inv64(uint64_t n) { return ip::inv64(n); }
uint32_t h_inv32(uint32_t n) { return ip::inv32(n); }
uint64_t h_mont_mul(uint64_t a, uint64_t b, uint64_t n) { return ip::mont_mul(a, b, n, ip::inv64(n)); }
uint64_t h_mod_dbl(uint64_t x, uint64_t n) { return ip::mod_dbl(x, n); }
void h_mont_setup(uint64_t n, uint64_t* out) {
  ip::Mont64 M = ip::mont64_setup(n);
  out[0] = M.q; out[1] = M.one; out[2] = M.mone; out[3] = ip::mont64_r2<0>(M);
  out[4] = M.ninv; out[5] = ip::mont64_r2<1>(M);
}
int h_sprp2_64(uint64_t n) {
  ip::Mont64 M = ip::mont64_setup(n);
  uint64_t d = n - 1; int s = ip::ctz64(d); d >>= s;
  int r0 = ip::sprp2_64<0>(M, d, s), r1 = ip::sprp2_64<1>(M, d, s);
  return r0 == r1 ? r0 : -1;
}
int h_sprp64(uint64_t n, uint64_t a) {  // a < n
  ip::Mont64 M = ip::mont64_setup(n);
  uint64_t d = n - 1; int s = ip::ctz64(d); d >>= s;
  uint64_t aR = ip::mont_mul_w(a, ip::mont64_r2<1>(M), n, M.q);
  uint64_t aR0 = ip::mont_mul(a, ip::mont64_r2<0>(M), n, M.ninv);
  if (aR0 != aR) return -1;
  int r1 = ip::sprp_tail64<1>(M, ip::mont_pow_binary<1>(M, aR, d), s);
  int r0 = ip::sprp_tail64<0>(M, ip::mont_pow_binary<0>(M, aR, d), s);
  return r1 == r0 ? r1 : -1;
}
uint32_t h_mont_mul32(uint32_t a, uint32_t b, uint32_t n) { return ip::mont_mul32(a, b, n, ip::inv32(n)); }
int h_sprp32(uint32_t n, uint32_t a) {
  ip::Mont32 M = ip::mont32_setup(n);
  uint32_t d = n - 1; int s = ip::ctz32(d); d >>= s;
  return ip::sprp32(M, a, d, s);
}
int h_td64(uint64_t n, int i) { return n * ip::kTdHost.inv64[i] <= ip::kTdHost.lim64[i]; }
int h_td32(uint32_t n, int i) { return (uint32_t)(n * ip::kTdHost.inv32[i]) <= ip::kTdHost.lim32[i]; }
uint32_t h_td_prime(int i) { return ip::kTdHost.p[i]; }
// The second trial-division stage over its first `groups` groups (-1: not a
// compiled group count).
int h_td2(uint64_t n, int groups) {
  switch (groups) {
    case 1: return ip::td2_divisible<1>(n, ip::kTd2Host);
    case 8: return ip::td2_divisible<8>(n, ip::kTd2Host);
    case 12: return ip::td2_divisible<12>(n, ip::kTd2Host);
    case 16: return ip::td2_divisible<16>(n, ip::kTd2Host);
    case 24: return ip::td2_divisible<24>(n, ip::kTd2Host);
    default: return -1;
  }
}
uint32_t h_td2_prime(int i) { return ip::kTd2Host.p[i]; }
int h_td_pair(uint64_t n) { return ip::td_pair_divisible(n, ip::kTdHost.inv32, ip::kTdHost.lim32); }
uint32_t h_mont_residue32(uint64_t n, uint32_t m) {
  return ip::mont_residue32((uint32_t)n, (uint32_t)(n >> 32), m, 0u - ip::inv32(m));
}
uint32_t h_td2_modulus(int g) { return ip::kTd2Host.m[g]; }
}

extern "C" {
uint64_t h_mont_mul_w(uint64_t a, uint64_t b, uint64_t n) {
  return ip::mont_mul_w(a, b, n, (uint32_t)(0u - ip::inv32((uint32_t)n)));
}
uint64_t h_mont_sqr_w(uint64_t a, uint64_t n) {
  return ip::mont_sqr_w(a, n, (uint32_t)(0u - ip::inv32((uint32_t)n)));
}
}

extern "C" {
uint64_t h_mont_sqr_h(uint64_t a, uint64_t n) { return ip::mont_sqr_h(a, n, ip::inv64(n)); }
}

extern "C" {
uint64_t h_mont_mul_f(uint64_t a, uint64_t b, uint64_t n) {
  return ip::mont_mul_f(a, b, n, (uint32_t)(0u - ip::inv32((uint32_t)n)));
}
uint64_t h_mont_sqr_f(uint64_t a, uint64_t n) {
  return ip::mont_sqr_f(a, n, (uint32_t)(0u - ip::inv32((uint32_t)n)));
}
}

// Stress check with an independent reference: REDC output r must satisfy
// r < n and r * 2^64 = a * b (mod n).  Returns the number of failures.
extern "C" uint64_t h_stress(uint64_t seed, uint64_t count, int variant) {
  uint64_t s = seed, bad = 0;
  auto next = [&s]() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (uint64_t i = 0; i < count; ++i) {
    uint64_t n = next() | 1;
    if (i % 4 == 0) n |= 1ull << 63;
    if (n < 3) n = 3;
    const uint64_t a = next() % n, b = (i % 3 == 0) ? a : next() % n;
    const uint32_t q = 0u - ip::inv32((uint32_t)n);
    const uint64_t ninv = ip::inv64(n);
    uint64_t r;
    switch (variant) {
      case 0: r = ip::mont_mul(a, b, n, ninv); break;
      case 1: r = ip::mont_mul_w(a, b, n, q); break;
      case 2: r = ip::mont_mul_f(a, b, n, q); break;
      case 3: r = ip::mont_sqr_f(a, n, q); break;
      case 4: r = ip::mont_sqr_h(a, n, ninv); break;
      default: r = ip::mont_sqr_w(a, n, q); break;
    }
    const uint64_t bb = (variant >= 3) ? a : b;
    const unsigned __int128 Rm = (((unsigned __int128)1) << 64) % n;
    const uint64_t lhs = (uint64_t)(((unsigned __int128)r * Rm) % n);
    const uint64_t rhs = (uint64_t)(((unsigned __int128)a * bb) % n);
    if (r >= n || lhs != rhs) ++bad;
  }
  return bad;
}

extern "C" {
int h_jacobi(int64_t a, uint64_t n) { return ip::jacobi_symbol(a, n); }
int h_jacobi_small(int32_t a, uint64_t n) { return ip::jacobi_small(a, n); }
int h_is_square(uint64_t n) { return ip::is_square64(n); }
int h_strong_lucas(uint64_t n) {
  const int r0 = ip::strong_lucas_selfridge<0>(n), r5 = ip::strong_lucas_selfridge<5>(n);
  return r0 == r5 ? r0 : -1;
}
}
