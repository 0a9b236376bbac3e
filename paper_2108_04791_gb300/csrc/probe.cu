// probe.cu -- integer-pipe throughput of this GPU (roofline denominators).
//
// Each kernel runs 8 independent dependency chains per thread over every SM
// at full occupancy, so issue rate rather than latency bounds it.  The
// operations are written as inline PTX so the compiler cannot fold them.
#include "arith.cuh"
#include "internal.h"

namespace ip {

constexpr int kChains = 8;
constexpr int kMontVariants = 10;
constexpr int kIters = 1024;

template <int kOp>
__global__ void __launch_bounds__(256) int_rate_kernel(uint32_t* sink, uint32_t seed,
                                                       unsigned long long* cycles) {
  uint32_t a[kChains], b[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = seed * (threadIdx.x + 1) + k;
    b[k] = seed ^ (k * 0x9E3779B9u);
  }
  const uint32_t m = seed | 1u;
  unsigned long long g0, g1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  long long t0 = clock64();
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (kOp == 0) {
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(m), "r"(b[k]));
      } else if (kOp == 1) {
        asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[k]) : "r"(m), "r"(b[k]));
      } else {
        // 32x32 + 64 -> 64: the 64-bit accumulator lives in (a, b)
        asm volatile(
            "{.reg .u64 t, c;\n\t"
            "mov.b64 c, {%0, %1};\n\t"
            "mad.wide.u32 t, %0, %2, c;\n\t"
            "mov.b64 {%0, %1}, t;}"
            : "+r"(a[k]), "+r"(b[k])
            : "r"(m));
      }
    }
  }
  long long t1 = clock64();
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc ^= a[k] ^ b[k];
  if (acc == 0x12345678u) sink[0] = acc;  // keeps the chains live
  // SM clock of this block's SM while it ran: cycles over global nanoseconds
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cycles[0] = (unsigned long long)(t1 - t0);
    cycles[1] = g1 - g0;
  }
}

// kVar 0: 128-bit product form (hi(ab) - hi(mn)); 1: word-level REDC with
// wide multiply-adds; 2: the word-level dedicated squaring; 3: squaring in
// the 128-bit form with one cross product; 4: 128-bit product with a PTX
// word-level REDC; 5: mont_mul(a, a); 6: fused product-scanning
// multiplication; 7: fused squaring; 8 and 9: multiplication and squaring
// of the 32-bit-word PTX form (mont_mul_c / mont_sqr_c).
template <int kVar>
__global__ void __launch_bounds__(256) mont_rate_kernel(uint64_t* sink, uint64_t seed) {
  uint64_t x[kChains];
  const uint64_t n = seed | (1ull << 63) | 1ull;
  const uint64_t ninv = inv64(n);
  const uint32_t q = 0u - inv32((uint32_t)n);
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (seed * (threadIdx.x + 1) + k) & ~(1ull << 63);
  for (int it = 0; it < kIters / 8; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (kVar == 0) x[k] = mont_mul(x[k], x[(k + 1) & (kChains - 1)], n, ninv);
      if (kVar == 1) x[k] = mont_mul_w(x[k], x[(k + 1) & (kChains - 1)], n, q);
      if (kVar == 2) x[k] = mont_sqr_w(x[k], n, q);
      if (kVar == 3) x[k] = mont_sqr_h(x[k], n, ninv);
      if (kVar == 4) x[k] = mont_mul_p(x[k], x[(k + 1) & (kChains - 1)], n, q);
      if (kVar == 5) x[k] = mont_mul(x[k], x[k], n, ninv);
      if (kVar == 6) x[k] = mont_mul_f(x[k], x[(k + 1) & (kChains - 1)], n, q);
      if (kVar == 7) x[k] = mont_sqr_f(x[k], n, q);
      if (kVar == 8) x[k] = mont_mul_c(x[k], x[(k + 1) & (kChains - 1)], n, ninv);
      if (kVar == 9) x[k] = mont_sqr_c(x[k], n, ninv);
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc ^= x[k];
  if (acc == 0x123456789ull) sink[0] = acc;
}

int measure_int_rates(int device, isprime_int_rates* out) {
  int ndev = 0;
  IP_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return set_error(ISPRIME_EINVAL, "device out of range");
  int prev = 0;
  IP_CUDA(cudaGetDevice(&prev));
  IP_CUDA(cudaSetDevice(device));
  int sms = 0, per_sm = 0;
  IP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  IP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_rate_kernel<0>, 256, 0));
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  uint32_t* sink = nullptr;
  unsigned long long* d_cyc = nullptr;
  IP_CUDA(cudaMalloc(&sink, 64));
  IP_CUDA(cudaMalloc(&d_cyc, 2 * sizeof(unsigned long long)));
  cudaEvent_t e0, e1;
  IP_CUDA(cudaEventCreate(&e0));
  IP_CUDA(cudaEventCreate(&e1));
  const double lane_ops = (double)grid * 256 * kIters * kChains;
  double rates[3] = {0, 0, 0};
  double mhz = 0;
  for (int op = 0; op < 3; ++op) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      IP_CUDA(cudaEventRecord(e0));
      if (op == 0) int_rate_kernel<0><<<grid, 256>>>(sink, 12345u + rep, d_cyc);
      if (op == 1) int_rate_kernel<1><<<grid, 256>>>(sink, 12345u + rep, d_cyc);
      if (op == 2) int_rate_kernel<2><<<grid, 256>>>(sink, 12345u + rep, d_cyc);
      IP_CUDA(cudaGetLastError());
      IP_CUDA(cudaEventRecord(e1));
      IP_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      IP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        if (op == 0) {
          unsigned long long cyc[2] = {0, 0};
          IP_CUDA(cudaMemcpy(cyc, d_cyc, sizeof cyc, cudaMemcpyDeviceToHost));
          mhz = cyc[1] ? 1e3 * (double)cyc[0] / (double)cyc[1] : 0.0;
        }
      }
    }
    rates[op] = lane_ops / (best * 1e-3);
  }
  double mont[kMontVariants] = {};
  for (int var = 0; var < kMontVariants; ++var) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      IP_CUDA(cudaEventRecord(e0));
      uint64_t* s64 = reinterpret_cast<uint64_t*>(sink);
      const uint64_t seed = 0x9E3779B97F4A7C15ull + rep;
      if (var == 0) mont_rate_kernel<0><<<grid, 256>>>(s64, seed);
      if (var == 1) mont_rate_kernel<1><<<grid, 256>>>(s64, seed);
      if (var == 2) mont_rate_kernel<2><<<grid, 256>>>(s64, seed);
      if (var == 3) mont_rate_kernel<3><<<grid, 256>>>(s64, seed);
      if (var == 4) mont_rate_kernel<4><<<grid, 256>>>(s64, seed);
      if (var == 5) mont_rate_kernel<5><<<grid, 256>>>(s64, seed);
      if (var == 6) mont_rate_kernel<6><<<grid, 256>>>(s64, seed);
      if (var == 7) mont_rate_kernel<7><<<grid, 256>>>(s64, seed);
      if (var == 8) mont_rate_kernel<8><<<grid, 256>>>(s64, seed);
      if (var == 9) mont_rate_kernel<9><<<grid, 256>>>(s64, seed);
      IP_CUDA(cudaGetLastError());
      IP_CUDA(cudaEventRecord(e1));
      IP_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      IP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) best = ms;
    }
    mont[var] = (double)grid * 256 * (kIters / 8) * kChains / (best * 1e-3);
  }
  out->mad_lo_u32 = rates[0];
  out->mad_hi_u32 = rates[1];
  out->mad_wide_u32 = rates[2];
  for (int v = 0; v < kMontVariants; ++v) out->mont_variant[v] = mont[v];
  out->sm_clock_mhz = mhz;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(d_cyc);
  cudaSetDevice(prev);
  return ISPRIME_OK;
}

}  // namespace ip
