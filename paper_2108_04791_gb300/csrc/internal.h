// internal.h -- library-private declarations shared by the .cu files.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/isprime.h"

namespace ip {

// Records the error text for isprime_last_error() and returns `status`.
int set_error(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// An NVTX range over the rest of the enclosing scope (entry points, batches,
// server dispatches): visible to Nsight tools, a few instructions otherwise.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
#define IP_NVTX(name) ::ip::NvtxRange ip_nvtx_range_(name)

#define IP_CUDA(call)                                     \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return ::ip::cuda_fail(e_, #call); \
  } while (0)

// Number of 32-bit queue counters (see Queues::counters).
constexpr int kQueueCounters = 8;

// Queue layout (device, per context).  Capacities are the chunk length, so a
// queue can hold every element of a chunk and never overflows.
struct Queues {
  uint64_t* q64_n = nullptr;    // values >= 2^32 that survived trial division
  uint32_t* q64_idx = nullptr;  // their indices within the chunk
  uint32_t* q64b = nullptr;     // positions in q64 that passed the base-2 test
  uint32_t* q32_n = nullptr;    // values in [S, 2^32) that survived trial division
  uint32_t* q32_idx = nullptr;
  // [0] q64 front size, [1] q64 back size (entries at capacity - 1,
  // capacity - 2, ...), [2] q64b size, [3] base-2 task counter, [4] q32 size,
  // [5..7] unused.  [0] and [1] form one 64-bit word (front + 2^32 back) that
  // classify advances with a single 64-bit atomic per warp for both regions
  // (two 32-bit atomics on one sector cost classify a third of its time).
  uint32_t* counters = nullptr;
  size_t capacity = 0;
};

// Batched path: one descriptor per array, and the batch header, in device
// memory (tile_begin = number of tiles of all earlier arrays).
struct BatchDesc {
  const uint64_t* in;
  uint8_t* out;
  uint64_t n;
  uint64_t tile_begin;
};
struct BatchHeader {
  uint64_t n_arrays;
  uint64_t total_tiles;
};

// State of one batched launch site: descriptor buffers, tile counter and the
// recorded graph.  A context owns one for its own calls; each server slot
// owns another, so batches on different streams never share them.
struct BatchState {
  void* d_batch = nullptr;           // BatchHeader + descriptors (device)
  void* h_batch = nullptr;           // pinned staging of the same
  size_t cap = 0;
  cudaEvent_t ev = nullptr;          // the last descriptor upload
  bool ev_valid = false;
  uint32_t* d_tile_counter = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t key = 0;
  unsigned grid = 0;
};
void batch_state_free(BatchState* b);

struct TimedLaunch {
  int kid;
  cudaEvent_t start, stop;
};

}  // namespace ip

struct isprime_ctx {
  int device = 0;
  int sm_count = 0;
  int smem_optin = 0;                // shared memory a block may opt into
  uint64_t sieve_limit = 0;
  uint32_t* d_sieve = nullptr;       // odd-only bitmap: bit j <-> 2j+1
  uint32_t* d_base_primes = nullptr; // odd primes < 2^16
  uint32_t* d_nprimes = nullptr;     // their count (device)
  uint32_t n_base_primes = 0;
  ip::Queues q;
  ip::Queues q2;                     // second queue set of the two-stream form (dual_stream)
  cudaStream_t dual_s = nullptr;     // its stream
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  isprime_tuning tune{};
  cudaEvent_t order_ev = nullptr;    // last use of the scratch queues
  bool order_ev_valid = false;
  std::mutex mu;
  std::mutex host_mu;  // serialises isprime_u64_host (staging buffers)
  // measurement
  bool timing = false;
  bool count_ops = false;            // isprime_count_ops: counting Miller-Rabin kernels
  std::vector<ip::TimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
  double kernel_ms[ISPRIME_K_COUNT] = {};
  uint64_t kernel_launches[ISPRIME_K_COUNT] = {};
  isprime_stats stats{};
  // end-to-end staging (host path)
  void* h_pin_in = nullptr;
  uint8_t* h_pin_out = nullptr;
  uint64_t* d_stage_in = nullptr;
  uint8_t* d_stage_out = nullptr;
  size_t stage_elems = 0;
  cudaStream_t copy_in = nullptr;    // host -> device copies of the host path
  cudaStream_t copy_out = nullptr;   // device -> host copies of the host path
  static constexpr int kStageSlots = 4;  // host path: staging buffers in flight
  cudaEvent_t stage_ev[3 * kStageSlots] = {};  // per staging slot: copied in, computed, copied out
  cudaEvent_t host_last = nullptr;   // end of the previous host-path call
  ip::BatchState batch;              // batched path of the context's own calls
  ip::Queues host_q[2];              // host path: one queue set per staging slot
  cudaStream_t host_s[2] = {};       // host path: one compute stream per staging slot
  // latency path (small.cu): results of inline calls land in mapped host memory
  std::mutex inline_mu;
  uint8_t* h_inline_out = nullptr;   // pinned, mapped, ISPRIME_HOST_INLINE_MAX bytes
  uint8_t* d_inline_out = nullptr;   // its device address
  cudaStream_t scalar_s = nullptr;   // stream of isprime_u64_scalar
  // double-path domain status: every f64 call adds its invalid elements to
  // d_status[0]; isprime_f64_sync_status takes it (into d_status[1]) after
  // the last f64 call (f64_ev), on status_s
  unsigned long long* d_status = nullptr;
  cudaEvent_t f64_ev = nullptr;
  bool f64_ev_valid = false;
  cudaStream_t status_s = nullptr;
  // window path (window.cu): min/max read-back and the window's bytes
  unsigned long long* d_mm = nullptr;
  unsigned long long* h_mm = nullptr;  // pinned
  uint64_t last_window_lo = 0, last_window_hi = 0;
  uint32_t fitted_window_ratio16 = 0;  // the autotuner's last crossover fit
  uint8_t* d_window = nullptr;
  size_t window_cap = 0;
};

namespace ip {

// The limit below which the array paths answer from the sieve: min(S, 2^k)
// for the tuned cutover k.
inline uint64_t sieve_cut(const isprime_ctx* c) {
  const uint64_t k = c->tune.sieve_cutover_log2 >= 32 ? (1ull << 32) : (1ull << c->tune.sieve_cutover_log2);
  return c->sieve_limit < k ? c->sieve_limit : k;
}

// Launch bracket: timing events + launch counting + error check.
int launch_begin(isprime_ctx* ctx, int kid, cudaStream_t s, TimedLaunch* tl);
int launch_end(isprime_ctx* ctx, cudaStream_t s, TimedLaunch* tl, const char* name);

// sieve.cu
int sieve_build(isprime_ctx* ctx, cudaStream_t s);
int ensure_base_primes(isprime_ctx* ctx, cudaStream_t s);

// range.cu
int range_run(isprime_ctx* ctx, uint64_t lo, uint64_t count, uint8_t* d_out, cudaStream_t s);
constexpr uint64_t kRangeChunkAlign = 1u << 15;  // integers per sieve segment
int sieve_count(isprime_ctx* ctx, cudaStream_t s, uint64_t* d_out);

// classify.cu
struct ClassifyArgs {
  const void* in;
  uint8_t* out;
  uint64_t n;                 // elements in this chunk
  const uint32_t* sieve;
  uint64_t sieve_limit;
  uint32_t ntd;
  uint64_t td_square;         // survivors of trial division below this are prime
  uint64_t* q64_n;
  uint32_t* q64_idx;
  uint32_t* q32_n;
  uint32_t* q32_idx;
  uint32_t* counters;
  unsigned long long* invalid;      // the caller's counter (nullable)
  unsigned long long* invalid_ctx;  // the context's own counter (nullable)
  uint32_t head;              // leading elements handled singly (alignment)
  uint32_t pair_store;        // 1 if out+head is 2-byte aligned (16-bit stores)
  uint32_t q64_cap;           // capacity of q64 (its back region ends there)
  uint32_t fold;              // fold level of the 64-bit trial division (0..2)
  uint32_t split;             // 1: 64-bit survivors split by s into q64's two regions
};
int launch_classify_u64(isprime_ctx* ctx, const ClassifyArgs& a, cudaStream_t s);
int launch_classify_f64(isprime_ctx* ctx, const ClassifyArgs& a, cudaStream_t s);

// mr.cu
// len: elements of the chunk just classified (bounds the queue lengths).
int launch_mr(isprime_ctx* ctx, const Queues& q, uint8_t* out, uint64_t len, cudaStream_t s);
// The operation counters of the counting kernels: [stage: base 2, six bases]
// [kind: squaring, product, 2^w step][warp issues, active lanes].
int op_counts_read(unsigned long long out[2][3][2], bool reset);

// Context-free launchers (explicit launch shape), used by noalloc.cu.
int launch_classify_u64_raw(const ClassifyArgs& a, unsigned grid, unsigned block, cudaStream_t s);
int launch_mr_raw(const Queues& q, uint8_t* out, bool with_mr32, unsigned grid, unsigned block,
                  cudaStream_t s);

// window.cu: the per-call choice of the window path for a u64 array of n
// values; *taken tells whether it ran (otherwise the queue path must).
int window_try(isprime_ctx* ctx, const uint64_t* d_in, uint8_t* d_out, size_t n, cudaStream_t s,
               bool* taken);
int array_minmax(isprime_ctx* ctx, const uint64_t* d_in, size_t n, cudaStream_t s, uint64_t* lo,
                 uint64_t* hi);
// The autotuner's crossover fit of the window path near the value `near`
// (arrays of up to n values); the context's tuning is unchanged.
int window_fit(isprime_ctx* ctx, uint64_t near, size_t n, cudaStream_t s, uint32_t* ratio16);

// Readers of the debug build's check words, one per translation unit with
// kernels (IP_CHECK_READER in device_common.cuh).
int check_read_classify(uint32_t* sites, uint64_t* count, bool reset);
int check_read_mr(uint32_t* sites, uint64_t* count, bool reset);
int check_read_batched(uint32_t* sites, uint64_t* count, bool reset);
int check_read_range(uint32_t* sites, uint64_t* count, bool reset);
int check_read_window(uint32_t* sites, uint64_t* count, bool reset);
int check_read_small(uint32_t* sites, uint64_t* count, bool reset);

// probe.cu
int measure_int_rates(int device, isprime_int_rates* out);

uint64_t td_square_for(uint32_t ntd);

// small.cu: one warp per element, one launch, no queues.
constexpr int kInlineMax = ISPRIME_HOST_INLINE_MAX;
int launch_small_u64(isprime_ctx* ctx, const uint64_t* d_in, uint8_t* d_out, size_t n,
                     cudaStream_t s);
int launch_small_f64(isprime_ctx* ctx, const double* d_in, uint8_t* d_out, size_t n,
                     unsigned long long* d_invalid, unsigned long long* d_invalid_ctx,
                     cudaStream_t s);
// A batch in one-warp-per-element form: d_descs[i].tile_begin holds the
// element prefix sum of array i (total elements in all arrays).
int launch_small_batched(isprime_ctx* ctx, const BatchDesc* d_descs, uint32_t n_arrays,
                         uint64_t total, cudaStream_t s);
// Host values in (n <= kInlineMax), host bytes out; takes ctx->inline_mu and
// ctx->mu itself and synchronises s.
int inline_run(isprime_ctx* ctx, const uint64_t* h_in, uint8_t* h_out, size_t n, cudaStream_t s);

// batched.cu
size_t batched_smem_bytes(uint32_t block, uint32_t tile);
// Runs one batch with the given launch-site state on stream s (no context
// ordering; the caller orders uses of `bs`).  A batch of at most warp_max
// elements in all runs as one warp-per-element launch.
int batched_run(isprime_ctx* ctx, BatchState* bs, const isprime_array* arrays, size_t n_arrays,
                uint64_t warp_max, cudaStream_t s);

}  // namespace ip
