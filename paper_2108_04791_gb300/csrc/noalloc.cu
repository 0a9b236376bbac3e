// noalloc.cu -- an entry point that never allocates memory.
//
// Some callers cannot allocate device memory at the moment they need a
// primality test: code running under an allocator that forbids cudaMalloc
// (a memory pool that owns the whole device), a callback or hook that must
// not block on the CUDA driver's allocation lock, or a process whose device
// memory is fully handed out in advance.  isprime_u64_noalloc serves them:
// it runs the classify and Miller-Rabin code of isprime_u64 (with the binary
// base-2 schedule, one queue region, and the six-base kernel without the
// variant that spreads short queues over threads) but keeps its work queues
// in one fixed array of device memory that is part of the library image
// (every GPU that loads the library holds it until the process exits), and
// it uses no sieve (values below 2^32 go through trial division and the
// 32-bit Miller-Rabin bases {2, 7, 61}).  It calls no cudaMalloc, cudaFree or
// any other allocating routine.
//
// The array's device address is looked up once per device and kept for the
// life of the process; a cudaDeviceReset (or anything else that destroys the
// device's primary context) invalidates it, so the entry point must not be
// used on a device after such a reset.
//
// Limits and sharing: at most kNoallocMaxElems elements per call; every
// call on a device uses the same array, which keeps the last call's
// contents, so calls whose GPU work overlaps (different streams, or
// threads, at the same time) race and must be ordered by the caller.
#include <mutex>

#include "internal.h"

namespace ip {

constexpr size_t kNoallocMaxElems = (size_t)1 << 20;  // ISPRIME_NOALLOC_MAX_ELEMS

// Queue storage for kNoallocMaxElems elements, 24 bytes each, plus the
// 32-bit queue counters (kQueueCounters of them) at the end: 24 MiB + 256 B.
constexpr size_t kNoallocQ64N = 0;                                   // u64 values
constexpr size_t kNoallocQ64Idx = kNoallocQ64N + 8 * kNoallocMaxElems;  // u32 indices
constexpr size_t kNoallocQ64B = kNoallocQ64Idx + 4 * kNoallocMaxElems;  // u32 positions
constexpr size_t kNoallocQ32N = kNoallocQ64B + 4 * kNoallocMaxElems;    // u32 values
constexpr size_t kNoallocQ32Idx = kNoallocQ32N + 4 * kNoallocMaxElems;  // u32 indices
constexpr size_t kNoallocCounters = kNoallocQ32Idx + 4 * kNoallocMaxElems;
constexpr size_t kNoallocBytes = kNoallocCounters + 256;
// classify advances counters[0..1] as one 64-bit word
static_assert(kNoallocCounters % 8 == 0, "queue counters must be 8-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Per-device set-up, done once by the first call on that device with the
// device current: the device address of the scratch array (host code only
// sees a host-side stand-in for the symbol) and the SM count.
struct NoallocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;
  int sm_count = 0;
};
static std::mutex g_noalloc_mu;
static NoallocDevice g_noalloc_dev[64];

static int noalloc_setup(int dev, NoallocDevice* out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
    d.scratch = static_cast<unsigned char*>(p);
    d.sm_count = sms;
    d.ready = true;
  }
  *out = d;
  return ISPRIME_OK;
}

}  // namespace ip

using namespace ip;

extern "C" int isprime_u64_noalloc(const uint64_t* d_in, uint8_t* d_out, size_t n,
                                   isprime_stream stream) {
  if (n == 0) return ISPRIME_OK;
  if (n > kNoallocMaxElems)
    return set_error(ISPRIME_EINVAL,
                     "isprime_u64_noalloc: n exceeds ISPRIME_NOALLOC_MAX_ELEMS (2^20); "
                     "split the array or use isprime_u64");
  if (!d_in || !d_out) return set_error(ISPRIME_EINVAL, "NULL pointer with n > 0");
  if ((uintptr_t)d_in % 8) return set_error(ISPRIME_EINVAL, "input not aligned to its element size");
  const uintptr_t a0 = (uintptr_t)d_in, a1 = a0 + n * 8, b0 = (uintptr_t)d_out, b1 = b0 + n;
  if (a0 < b1 && b0 < a1) return set_error(ISPRIME_EINVAL, "output overlaps input");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return set_error(ISPRIME_EINVAL, "device out of range");
  NoallocDevice d;
  int st = noalloc_setup(dev, &d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;

  Queues q;
  q.q64_n = reinterpret_cast<uint64_t*>(d.scratch + kNoallocQ64N);
  q.q64_idx = reinterpret_cast<uint32_t*>(d.scratch + kNoallocQ64Idx);
  q.q64b = reinterpret_cast<uint32_t*>(d.scratch + kNoallocQ64B);
  q.q32_n = reinterpret_cast<uint32_t*>(d.scratch + kNoallocQ32N);
  q.q32_idx = reinterpret_cast<uint32_t*>(d.scratch + kNoallocQ32Idx);
  q.counters = reinterpret_cast<uint32_t*>(d.scratch + kNoallocCounters);
  q.capacity = kNoallocMaxElems;
  // The counters keep the previous call's values: start them at zero.
  e = cudaMemsetAsync(q.counters, 0, kQueueCounters * sizeof(uint32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");

  constexpr uint32_t kTdPrimes = 15;  // 3..53, as in the default tuning
  ClassifyArgs a;
  a.in = d_in;
  a.out = d_out;
  a.n = n;
  a.sieve = nullptr;
  a.sieve_limit = 0;
  a.ntd = kTdPrimes;
  a.td_square = td_square_for(kTdPrimes);
  a.q64_n = q.q64_n;
  a.q64_idx = q.q64_idx;
  a.q32_n = q.q32_n;
  a.q32_idx = q.q32_idx;
  a.counters = q.counters;
  a.invalid = nullptr;
  a.invalid_ctx = nullptr;
  a.head = ((uintptr_t)d_in % 16) ? 1u : 0u;
  a.pair_store = (((uintptr_t)(d_out + a.head)) % 2 == 0) ? 1u : 0u;
  a.q64_cap = (uint32_t)q.capacity;
  a.fold = 0;
  a.split = 0;
  const unsigned block = 256;
  const uint64_t npairs = (n - a.head) / 2;
  const uint64_t want = (npairs + 4 * block - 1) / (4 * block);  // 4 pairs per thread per tile
  const uint64_t cap = (uint64_t)d.sm_count * 8;
  const unsigned grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  if ((st = launch_classify_u64_raw(a, grid, block, s))) return st;
  return launch_mr_raw(q, d_out, /*with_mr32=*/true, (unsigned)d.sm_count * 8, 128, s);
}
