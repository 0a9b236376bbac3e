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
  out[0] = M.ninv; out[1] = M.one; out[2] = M.mone; out[3] = ip::mont64_r2(M);
}
int h_sprp2_64(uint64_t n) {
  ip::Mont64 M = ip::mont64_setup(n);
  uint64_t d = n - 1; int s = ip::ctz64(d); d >>= s;
  return ip::sprp2_64(M, d, s);
}
int h_sprp64(uint64_t n, uint64_t a) {  // a < n
  ip::Mont64 M = ip::mont64_setup(n);
  uint64_t d = n - 1; int s = ip::ctz64(d); d >>= s;
  uint64_t aR = ip::mont_mul(a, ip::mont64_r2(M), n, M.ninv);
  return ip::sprp_tail64(M, ip::mont_pow_binary(M, aR, d), s);
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
}
