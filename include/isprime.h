/*
 * isprime.h -- C ABI of the GB300 elementwise primality library.
 *
 * The operation (paper: "Improving MATLAB's isprime performance without
 * arbitrary-precision arithmetic", Sec. 1): given an array N, return an
 * array of the same length whose element i is 1 if N[i] is prime and 0
 * otherwise.  Values are unsigned 64-bit integers (uint64 path), or doubles
 * that hold integers up to 2^53 (double path; Sec. 8.1 uses double up to
 * 2^53 and uint64 above).  The result is exact for every value: small values
 * are answered by a device-resident sieve (Sec. 6.1.3), the rest by trial
 * division by small primes (Sec. 6.1.2) and deterministic Miller-Rabin with
 * the seven bases of Eq. 4 (Sec. 2.1) in 64-bit Montgomery arithmetic, or the
 * bases {2, 7, 61} below 2^32 (optionally base 2 and a strong Lucas test,
 * the Baillie-PSW test of Sec. 10.1).  Short arrays and single values take a
 * one-launch path with one warp per value.
 *
 * Conventions for every entry point:
 *   - Return value: ISPRIME_OK (0) or a negative isprime_status.  The text of
 *     the most recent error on the calling thread is isprime_last_error().
 *   - Pointers named d_* are device pointers (cudaMalloc'd or torch storage on
 *     the context's device); h_* are host pointers.  The caller owns every
 *     buffer it passes; the library owns its contexts (resident sieve, work
 *     queues, staging buffers) and frees them in isprime_ctx_destroy.
 *   - Device entry points are asynchronous on `stream` (a cudaStream_t; NULL
 *     is the legacy default stream).  Outputs are valid once the stream has
 *     synchronised.  Calls on one context from several streams are ordered
 *     by the library (they share the context's work queues).
 *   - n == 0 is a no-op returning ISPRIME_OK.  A NULL pointer with n > 0, an
 *     input pointer that is not aligned to its element type, or an output
 *     range that overlaps the input range gives ISPRIME_EINVAL and launches
 *     nothing.
 *   - Output bytes are exactly 0 or 1, in input order.
 */
#ifndef ISPRIME_H_
#define ISPRIME_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ISPRIME_OK = 0,
  ISPRIME_EINVAL = -1,    /* bad argument (NULL, misaligned, overlap, range) */
  ISPRIME_ENOMEM = -2,    /* device or pinned-host allocation failed */
  ISPRIME_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
  ISPRIME_EDOMAIN = -4,   /* double input held values that are not integers in [0, 2^53] */
  ISPRIME_ETIMEDOUT = -5, /* a bounded wait ran out */
  ISPRIME_EBUSY = -6      /* request larger than the server's memory budget */
} isprime_status;

typedef struct isprime_ctx isprime_ctx;
typedef struct CUstream_st *isprime_stream; /* same type as cudaStream_t */

/* Launch and algorithm parameters of a context.  Results never depend on
 * them; only speed does. */
typedef struct {
  uint32_t classify_block; /* threads per block of the classify kernel (32..1024, multiple of 32) */
  uint32_t mr_block;       /* threads per block of the Miller-Rabin kernels (32..256, multiple of 32) */
  uint32_t blocks_per_sm;  /* grid = SMs x blocks_per_sm for grid-stride kernels (1..32) */
  uint32_t td_primes;      /* odd primes 3, 5, 7, ... used for trial division (0..53) */
  uint32_t chunk_log2;     /* elements per internal chunk = 2^chunk_log2 (16..28) */
  uint32_t mont_impl;      /* 64-bit Montgomery formulation of the six-base kernel: 0 128-bit
                              product (squaring with one cross product), 1 word-level, 2 128-bit
                              product with PTX word-level reduction, 3 fused product scanning,
                              4 128-bit multiply with fused squaring, 5 128-bit product with
                              squaring as a general multiply, 6 128-bit form in 32-bit words
                              (PTX, wide products and carry chains, no m0 n0 product),
                              7 formulation 6 with the partial sums carried in the wide
                              products' 64-bit addends, 8 formulation 7 with squaring as a
                              general multiply, 9 formulation 6 with its final "+ n when
                              negative" as multiply-adds (multiply pipe) instead of ANDs and
                              adds (ALU pipe; default) */
  uint32_t mont_impl_base2;/* the same choice for the base-2 kernel (0..9) */
  uint32_t batch_block;    /* threads per block of the batched kernel (32..256, multiple of 32; the
                              shared memory of batch_block and batch_tile_log2 must fit a block) */
  uint32_t batch_tile_log2;/* elements per tile of the batched kernel = 2^batch_tile_log2 (8..14) */
  uint32_t batch_blocks_per_sm; /* cap on resident batched blocks per SM (0 = occupancy limit) */
  uint32_t base2_window;   /* base-2 exponentiation: 0 binary with a doubling per set bit;
                              1 4-bit windows, x 2^w mod n as x 2^w - q n with q estimated
                              from a single-precision reciprocal of n (default); 2 the same
                              windows with q estimated in integers (one high multiply by a 32-bit
                              reciprocal of n); 4 4-bit windows, x 2^w R mod n by a Montgomery
                              product with a table of 2^w R in shared memory.  Modes 1 and 2
                              take the second trial stage, finishing in place and (mode 1) two
                              survivors per thread (with the second trial stage for td2_groups
                              16 and 24) */
  uint32_t rest_test;      /* after base 2: 0 the six remaining bases of Eq. 4 (default), 1 the
                              strong Lucas test with Selfridge's parameters (Baillie-PSW).
                              Both are exact below 2^64; 1 rests on the published search
                              finding no Baillie-PSW pseudoprime below 2^64. */
  uint32_t small_max;      /* arrays of at most small_max elements take the one-launch latency
                              path (one warp per element, no queues; 0..2^20, 0 = never) */
  uint32_t compact_min;    /* survivor compaction after base 2: a warp with at least
                              compact_min survivors finishes them in place (the rest_test
                              stage run by the same warp) instead of appending them to the
                              survivor queue; 0..33, 33 = always compact.  In-place finishing
                              needs base2_window 1 or 4 (with 0 the survivors are always compacted);
                              with 0 or 1 every survivor is finished in place and the six-base
                              kernel is not launched */
  uint32_t sieve_cutover_log2; /* sieve / Miller-Rabin cutover of the array paths: the resident
                              sieve answers n < min(S, 2^k); values from there up to 2^32 take
                              trial division and the 32-bit Miller-Rabin test (0..32) */
  uint32_t serve_short_max;/* a server created on the context batches requests of at most this
                              many elements apart from longer ones, as one-launch warp batches
                              on high-priority streams (0..2^20) */
  uint32_t td_fold;        /* trial division of 64-bit values by the primes 3..53 (td_primes 15):
                              0 every prime by the 64-bit multiply-by-inverse test; 1 the primes
                              dividing 2^32-1, 2^24-1 and 2^20-1 (3, 5, 7, 11, 13, 17, 31, 41)
                              by the 32-bit test on a sum of chunks of n that is congruent to n
                              modulo that number; 2 also 29 and 43 by 2^28-1; 3 every prime by
                              the 32-bit test on one of two residues of n, modulo
                              29*31*41*43*47*53 and 3*5*7*11*13*17*19*23*37 (each below 2^32,
                              one Montgomery reduction step each) */
  uint32_t base2_split;    /* 1: 64-bit survivors with n = 3 (mod 4) (s = 1 in n-1 = 2^s d) are
                              queued apart from the others, so the base-2 kernel's warps of those
                              run no strong-test tail; 0: one queue */
  uint32_t base2_ilp;      /* survivors per thread in the base-2 kernel (1 or 2; 2 takes effect
                              with base2_window 1, mont_impl_base2 6 or 9 and compact_min 33) */
  uint32_t rest_window;    /* window bits of the six-base exponentiations (3 or 4; 3 takes effect
                              with mont_impl 6 or 9) */
  uint32_t window_ratio16; /* per-call path choice of the uint64 array entry points (Sec. 6.2's
                              choice between sieving up to max(N) and testing each element):
                              0 never (default); otherwise a call of at least 2^16 values reads
                              the array's min and max (one reduction kernel; the call waits for
                              it) and, when max >= S, W = max - min + 1 <= 2^30 and
                              16 W <= window_ratio16 * n, classifies every integer of [min, max]
                              with the range kernels and gathers the array's bytes from that
                              window instead of running the queue path.  0..4096; the
                              autotuner measures the crossover on this GPU */
  uint32_t base2_blocks_per_sm; /* cap on resident blocks per SM of the base-2 kernel (a single
                              wave of persistent blocks; 0 = as many as fit, 1..32) */
  uint32_t pdl;            /* 1: the Miller-Rabin kernels are launched with programmatic stream
                              serialisation, so a launch overlaps the end of the kernel before it
                              (each waits for that kernel before reading the queues; default);
                              0: plain stream order */
  uint32_t td2_groups;     /* second trial-division stage: the base-2 kernel first tests its
                              queue's values against the odd primes after 53 in this many
                              groups of three (0, 8, 12, 16 or 24: primes up to 173, 239, 311,
                              457) and runs the base-2 test only on those no prime divides,
                              staged per warp so that the tests run on full warps (with
                              base2_window 1, base2_ilp 1, formulations 6 and 9); 0: off */
  uint32_t dual_stream;    /* 1: arrays of at least 2^20 values run as at least two chunks that
                              alternate between the caller's stream and a second stream of the
                              context with its own queues (fork and join by events, so the call
                              keeps the caller's stream order); 0: one stream */
  uint32_t host_chunk_log2;  /* isprime_u64_host: chunks of at most 2^host_chunk_log2 values
                              (and at most 2^chunk_log2), 16..24, default 22 */
  uint32_t inplace_max_log2; /* chunks of at most 2^inplace_max_log2 values run as if
                              compact_min were 1 (base2_window 1 or 4): the base-2 kernel's
                              warps finish their own passers and the six-base kernel is not
                              launched; 0..24, 0 = never */
  uint32_t serve_long_log2;  /* a server created on the context closes a batch of long requests
                              once it holds 2^serve_long_log2 values (its first request may be
                              larger); 16..28, default 24 */
  uint32_t rest_ilp;       /* six-base kernel on long queues with rest_window 3: the bases one
                              at a time (1) or in pairs, two exponentiations interleaved per
                              thread (2, default) */
} isprime_tuning;

/* Per-context counters since creation (or the last reset). */
typedef struct {
  uint64_t calls;          /* API calls that launched work */
  uint64_t elements;       /* elements classified */
  uint64_t kernel_launches;/* kernels launched by the library */
  uint64_t sieve_limit;    /* S: values below S are answered by the sieve */
  uint64_t scratch_bytes;  /* device memory held by the context */
  uint64_t window_calls;   /* calls that took the window path (window_ratio16) */
} isprime_stats;

/* ---------------------------------------------------------------- contexts */

/* Creates a context on `device`: builds the odd-only sieve bitmap for
 * [0, sieve_limit) on the GPU (S/16 bytes; Sec. 6.1.3's sieve up to the array
 * maximum, kept resident) and allocates the work queues.  sieve_limit must be
 * 0 (no sieve) or a multiple of 2^20 no larger than 2^32; ISPRIME_SIEVE_DEFAULT
 * selects 2^32.  Blocks until the sieve is built.  *out receives the
 * context; the caller destroys it with isprime_ctx_destroy. */
#define ISPRIME_SIEVE_DEFAULT ((uint64_t)-1)
int isprime_ctx_create(int device, uint64_t sieve_limit, isprime_ctx **out);

/* Synchronises the context's device work and frees everything it owns. */
int isprime_ctx_destroy(isprime_ctx *ctx);

/* The per-device default context used by the entry points without _ctx,
 * created on first use (sieve limit 2^32) and kept until process exit. */
int isprime_default_ctx(int device, isprime_ctx **out);

int isprime_ctx_get_tuning(const isprime_ctx *ctx, isprime_tuning *out);
/* The parameters a new context starts with (no device is touched). */
int isprime_tuning_defaults(isprime_tuning *out);
/* Validates and installs new parameters (ISPRIME_EINVAL if out of range). */
int isprime_ctx_set_tuning(isprime_ctx *ctx, const isprime_tuning *t);
int isprime_ctx_stats(const isprime_ctx *ctx, isprime_stats *out);

/* ------------------------------------------------------------- the hot path */

/* out[i] = isprime(in[i]) for i < n (Sec. 1; Sec. 2 for 64-bit values).
 * d_in: n uint64 values, 8-byte aligned.  d_out: n bytes.  Uses the default
 * context of the current device. */
int isprime_u64(const uint64_t *d_in, uint8_t *d_out, size_t n, isprime_stream stream);
int isprime_u64_ctx(isprime_ctx *ctx, const uint64_t *d_in, uint8_t *d_out, size_t n,
                    isprime_stream stream);

/* Double path (Sec. 8.1): element i is valid when it is finite, >= 0,
 * integral and <= 2^53; valid elements are classified as integers, invalid
 * ones give 0.  If d_invalid is not NULL, the number of invalid elements is
 * also added to the device counter *d_invalid (the caller zeroes it and reads
 * it after synchronising).  Whether or not d_invalid is given, the count is
 * added to the context's own counter, which isprime_f64_sync_status reports
 * as ISPRIME_EDOMAIN.  The double-path calls of one context run one after
 * another on the GPU (each waits for the previous one's kernels), whatever
 * streams they are made on.  isprime_f64 uses the current device's default
 * context (isprime_default_ctx). */
int isprime_f64(const double *d_in, uint8_t *d_out, size_t n, unsigned long long *d_invalid,
                isprime_stream stream);
int isprime_f64_ctx(isprime_ctx *ctx, const double *d_in, uint8_t *d_out, size_t n,
                    unsigned long long *d_invalid, isprime_stream stream);

/* Domain status of the double path (Sec. 8.1 stores integers in doubles only
 * up to 2^53; the paper does not say what other doubles give, and this
 * library answers 0 for them and reports them here).  Waits until every
 * double-path call made on ctx before this call has run, then takes the
 * context's count of invalid elements since the previous status call (or the
 * context's creation) and resets it to 0.  *count (nullable) receives it.
 * Returns ISPRIME_EDOMAIN if it was not 0, else ISPRIME_OK; ISPRIME_EINVAL
 * for a NULL ctx; ISPRIME_ECUDA if a CUDA call failed.  Synchronous. */
int isprime_f64_sync_status(isprime_ctx *ctx, unsigned long long *count);

/* Range form: d_out[i] = isprime(lo + i) for i < count, with no input array
 * (the incrementing sequences 1:N of Sec. 6.1.3 / Table 3 and the windows of
 * consecutive integers of Table 5).  Requires lo + count <= 2^64.  Values
 * below the context's sieve limit are read from the resident bitmap; the
 * rest are sieved in shared memory by the odd primes below 2^16 and the
 * survivors above 65537^2 finish with the 64-bit Miller-Rabin kernels.
 * Asynchronous on `stream`. */
int isprime_range(isprime_ctx *ctx, uint64_t lo, uint64_t count, uint8_t *d_out,
                  isprime_stream stream);

/* One array of a batch: n values at d_in (8-byte aligned), n bytes at d_out. */
typedef struct {
  const uint64_t *d_in;
  uint8_t *d_out;
  uint64_t n;
} isprime_array;

/* Batched form: classifies every array of `arrays` (a host array of
 * n_arrays descriptors) in one persistent kernel launch, replayed from a
 * CUDA graph that the context records on first use.  Results are identical
 * to calling isprime_u64_ctx on each array.  Arrays may have any lengths
 * (including 0); no array's output may overlap any array's input or output.
 * Asynchronous on `stream`; the descriptors are copied before return. */
int isprime_u64_batched(isprime_ctx *ctx, const isprime_array *arrays, size_t n_arrays,
                        isprime_stream stream);

/* Autotuner: chooses the context's tuning (every field that affects only
 * speed) by timing the caller's device sample d_sample (n values) on this
 * GPU; d_scratch_out is n bytes of device memory for the outputs.  mode
 * ISPRIME_TUNE_PLAIN tunes isprime_u64_ctx, ISPRIME_TUNE_BATCHED tunes
 * isprime_u64_batched (the sample is cut into ragged arrays).  Coordinate
 * descent over candidate values, best of three timed runs per candidate.
 * If cache_path is not NULL and holds a result for this GPU, runtime
 * version, sample size and mode, that result is installed without timing;
 * otherwise the result is appended to the file.  *out (nullable) receives
 * the installed tuning.  Synchronous. */
#define ISPRIME_TUNE_PLAIN 0
#define ISPRIME_TUNE_BATCHED 1
int isprime_autotune(isprime_ctx *ctx, const uint64_t *d_sample, uint8_t *d_scratch_out, size_t n,
                     int mode, const char *cache_path, isprime_tuning *out);
/* Writes "field=value,..." for every tuning field into buf (cap bytes). */
int isprime_tuning_format(const isprime_tuning *t, char *buf, size_t cap);

/* End-to-end form for host buffers: copies h_in to the device in chunks
 * (through the context's staging buffers), classifies each chunk on the
 * context's own streams while the next one is copied, copies the bytes back
 * into h_out and returns when h_out holds every result.  `stream` carries only
 * calls of at most ISPRIME_HOST_INLINE_MAX values.  h_in and h_out may be
 * pageable or pinned (pinned memory gives asynchronous copies). */
int isprime_u64_host(isprime_ctx *ctx, const uint64_t *h_in, uint8_t *h_out, size_t n,
                     isprime_stream stream);

/* Latency path for one value (the paper's scalar calls, Sec. 1 and Table 4):
 * *result = isprime(value).  The value travels in the kernel's parameters and
 * the answer comes back through mapped pinned host memory, so a call is one
 * kernel launch (one warp: trial division spread over the lanes, the seven
 * bases of Eq. 4 on seven lanes at once) and one synchronisation of the
 * context's own stream.  Synchronous; thread-safe. */
int isprime_u64_scalar(isprime_ctx *ctx, uint64_t value, uint8_t *result);

/* isprime_u64_host sends arrays of at most ISPRIME_HOST_INLINE_MAX values
 * the same way (no copies); longer arrays take the staged, pipelined path. */
#define ISPRIME_HOST_INLINE_MAX 256

/* Allocation-free variant of isprime_u64 (the paper has no counterpart;
 * this exists for callers that cannot allocate device memory when they need
 * the test -- e.g. code running under an allocator that owns all device
 * memory, or a hook that must not take the CUDA driver's allocation lock).
 * Same inputs, outputs and results as isprime_u64, but the work queues live
 * in one fixed array of ISPRIME_NOALLOC_SCRATCH_BYTES of device memory that
 * is part of the library image (every GPU that loads the library holds it
 * until exit); no sieve is used.  Calls no cudaMalloc, cudaFree or other
 * allocating routine.  n > ISPRIME_NOALLOC_MAX_ELEMS gives ISPRIME_EINVAL.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not call
 * this entry point on a device after cudaDeviceReset (or anything else that
 * destroys the device's primary context), which invalidates the address.
 * All calls on a device share the array: calls whose GPU work overlaps race,
 * so the caller must order them (one stream, or events). */
#define ISPRIME_NOALLOC_MAX_ELEMS ((size_t)1 << 20)
#define ISPRIME_NOALLOC_SCRATCH_BYTES ((size_t)24 * ((size_t)1 << 20) + 256)
int isprime_u64_noalloc(const uint64_t *d_in, uint8_t *d_out, size_t n, isprime_stream stream);

/* Number of primes below the context's sieve limit S, counted on the device
 * from the resident bitmap (pi(S); 0 when S == 0).  Synchronous. */
int isprime_sieve_count(isprime_ctx *ctx, uint64_t *out);

/* ------------------------------------------- sharding a job across devices */
/* Every element is independent (Sec. 1: element i of the result depends on
 * N[i] alone), so one job splits across devices with no exchange of data
 * between them.  These helpers decide which device takes which part; each
 * device then runs the plain, batched or served entry points on its part with
 * its own context.  Host only: no device is touched, no context is needed. */

/* Contiguous split of n elements into n_shards ranges whose sizes differ by
 * at most one (the first n mod n_shards ranges take one more): shard s takes
 * [begin[s], begin[s+1]).  begin: caller-owned, n_shards + 1 entries.
 * n_shards == 0 or begin == NULL: ISPRIME_EINVAL. */
int isprime_plan_contiguous(uint64_t n, uint32_t n_shards, uint64_t *begin);

/* Whole arrays of a batch, sizes[i] elements each, to n_shards by
 * longest-processing-time first: arrays in decreasing size (equal sizes in
 * index order), each to the shard with the least total so far (ties to the
 * lower shard index).  Every shard's total is at most the mean total plus the
 * largest array, and the largest total at most 4/3 of the best possible.
 * owner[i] receives the shard of array i; load[s] (nullable, n_shards
 * entries) the elements of shard s.  Caller-owned arrays.  n_arrays == 0
 * only fills load with zeros.  NULL sizes or owner with n_arrays > 0, or
 * n_shards == 0: ISPRIME_EINVAL. */
int isprime_plan_batched(const uint64_t *sizes, size_t n_arrays, uint32_t n_shards,
                         uint32_t *owner, uint64_t *load);

/* Served requests across devices: *device receives the index of the device
 * with the least outstanding work (outstanding[d]: elements admitted to
 * device d and not yet finished), ties to the lower index.  n_devices == 0 or
 * a NULL pointer: ISPRIME_EINVAL. */
int isprime_route_least_loaded(const uint64_t *outstanding, uint32_t n_devices,
                               uint32_t *device);

/* One host-array job on several devices: h_in (n values) is split by
 * isprime_plan_contiguous into n_devices ranges, range k runs on device
 * devices[k] through isprime_u64_host with that device's default context, in
 * a host thread of its own, and the results land in h_out in input order.
 * Nothing is exchanged between devices.  A device may appear more than once
 * (its ranges then run one after another).  Synchronous; returns the first
 * shard's error, if any.  n_devices == 0, a NULL pointer with n > 0 or a
 * device out of range: ISPRIME_EINVAL, before any device is touched. */
int isprime_u64_host_multi(const int *devices, uint32_t n_devices, const uint64_t *h_in,
                           uint8_t *h_out, size_t n);

/* ---------------------------------------------------------------- serving */

/* A continuous-batching server on one context.  Requests (host arrays) are
 * admitted as they arrive; a dispatcher thread groups the requests waiting
 * at that moment into a batch whenever one of n_slots stream slots and
 * enough of the device-memory budget (9 bytes per element, rounded to 256 B
 * per buffer) are free, and runs copy-in / one batched launch / copy-out on
 * that slot.  Batches on different slots overlap on the GPU.  The context's
 * sieve stays resident and is shared by all batches. */
typedef struct isprime_server isprime_server;

typedef struct {
  uint64_t requests;   /* completed requests since creation or the last reset */
  uint64_t elements;   /* their elements */
  uint64_t batches;    /* batches launched */
  double p50_ms;       /* latency percentiles: completion time - submit time */
  double p99_ms;
  double mean_ms;
  double max_ms;
  double span_s;       /* first submit to last completion */
  double tests_per_s;  /* elements / span_s */
  uint64_t short_requests; /* requests of at most small_max elements (batched apart) */
  double p50_short_ms; /* latency percentiles of the short requests */
  double p99_short_ms;
  double p50_long_ms;  /* and of the others */
  double p99_long_ms;
} isprime_server_stats;

/* Allocates a device arena of mem_budget_bytes and starts the server's two
 * threads.  n_slots in [1, 16]. */
int isprime_server_create(isprime_ctx *ctx, size_t mem_budget_bytes, int n_slots,
                          isprime_server **out);
/* Admits a request and returns at once with *ticket.  h_in (n values,
 * 8-byte aligned) and h_out (n bytes) must stay valid until the ticket is
 * waited for; pinned memory gives asynchronous copies.  ISPRIME_EBUSY if the
 * request alone needs more device memory than the budget. */
int isprime_server_submit(isprime_server *srv, const uint64_t *h_in, uint8_t *h_out, size_t n,
                          uint64_t *ticket);
/* Waits for a ticket (timeout_ms < 0: no limit).  ISPRIME_OK once h_out holds
 * the result (the ticket is then released); ISPRIME_ETIMEDOUT if it did not
 * finish in time (the ticket stays valid); ISPRIME_EINVAL for an unknown
 * ticket. */
int isprime_server_wait(isprime_server *srv, uint64_t ticket, int timeout_ms);
int isprime_server_get_stats(isprime_server *srv, isprime_server_stats *out);
int isprime_server_reset_stats(isprime_server *srv);
/* Stops admitting, finishes every admitted request, joins the threads and
 * frees the server (not the context). */
int isprime_server_destroy(isprime_server *srv);

/* ------------------------------------------------------------ measurement */

/* Kernel identifiers for the timing records. */
enum {
  ISPRIME_K_SIEVE_BASE = 0,
  ISPRIME_K_SIEVE_SEGMENT = 1,
  ISPRIME_K_CLASSIFY_U64 = 2,
  ISPRIME_K_CLASSIFY_F64 = 3,
  ISPRIME_K_MR64_BASE2 = 4,
  ISPRIME_K_MR64_REST = 5,
  ISPRIME_K_MR32 = 6,
  ISPRIME_K_SIEVE_COUNT = 7,
  ISPRIME_K_BATCHED = 8,
  ISPRIME_K_RANGE = 9,
  ISPRIME_K_SMALL = 10,
  ISPRIME_K_COUNT = 11
};

typedef struct {
  double total_ms;   /* summed CUDA-event duration of the kernel's launches */
  uint64_t launches; /* launches recorded */
} isprime_kernel_time;

/* While enabled, every kernel launch of the context is bracketed by CUDA
 * events recorded on the launching stream.  isprime_timing_read synchronises
 * the recorded events and returns per-kernel totals for the ISPRIME_K_COUNT
 * kernels (array `out` of that length); reset clears them. */
int isprime_timing_enable(isprime_ctx *ctx, int on);
int isprime_timing_read(isprime_ctx *ctx, isprime_kernel_time *out, int count);
int isprime_timing_reset(isprime_ctx *ctx);

/* Integer-pipe throughput of this GPU, measured by kernels of independent
 * dependency chains (8 per thread, all SMs, full occupancy).  Rates are lane
 * operations per second; sm_clock_mhz is the SM clock seen during the
 * measurement (clock64 cycles / event time).  Synchronous; used to state
 * the integer-pipe roofline of the Miller-Rabin kernels. */
typedef struct {
  double mad_lo_u32;     /* mad.lo.u32 */
  double mad_hi_u32;     /* mad.hi.u32 */
  double mad_wide_u32;   /* mad.wide.u32 (32x32+64 -> 64) */
  /* 64-bit Montgomery operations per second, by formulation:
   * [0] multiply, 128-bit product and hi(ab) - hi(mn) REDC
   * [1] multiply, word-level REDC with wide multiply-adds
   * [2] squaring, word-level
   * [3] squaring, 128-bit form with one cross product
   * [4] multiply, 128-bit product with a word-level REDC in PTX carry chains
   * [5] squaring as a general multiply of [0]
   * [6] multiply, fused product-scanning form (wide multiply-adds carry all carries)
   * [7] squaring, fused form
   * [8] multiply, 32-bit-word PTX form without the m0 n0 product (formulation 6)
   * [9] squaring, the same form */
  double mont_variant[10];
  double sm_clock_mhz;
} isprime_int_rates;
int isprime_measure_int_rates(int device, isprime_int_rates *out);

/* Executed Montgomery operations of the two 64-bit Miller-Rabin stages, as
 * issued by the GPU: each pair is [warp-level issues, active lanes summed
 * over those issues].  A warp issue occupies all 32 lanes of the integer
 * pipes whatever the number of active lanes, so 32 x issues is the lane work
 * paid and the active-lane sum the part that carried a value; the canonical
 * count of the method (binary left-to-right schedule, Sec. 2.4) is smaller
 * than either by the warp-uniform padding of the schedules and the
 * window-table products. */
typedef struct {
  uint64_t elements;
  uint64_t base2_squarings[2]; /* base-2 stage: Montgomery squarings */
  uint64_t base2_products[2];  /* Montgomery products (window table, mode 4) */
  uint64_t base2_steps[2];     /* x 2^w mod n window steps (mode 1) */
  uint64_t rest_squarings[2];  /* six-base stage: squarings (incl. R^2 setup) */
  uint64_t rest_products[2];   /* products (base conversion, tables, windows) */
} isprime_op_counts;
/* Runs isprime_u64_ctx's queue path once on d_in (n values; d_out receives
 * the results) with the Miller-Rabin kernels built to count their
 * operations (formulation 6 plus counting; slower), synchronously, and
 * returns the counts.  Measurement only: no other thread may use ctx during
 * the call.  Argument errors as isprime_u64_ctx. */
int isprime_count_ops(isprime_ctx *ctx, const uint64_t *d_in, uint8_t *d_out, size_t n,
                      isprime_op_counts *out);

/* Bounds checks of the debug build of the library (built with
 * IP_DEBUG_CHECKS, `python -m paper_2108_04791_gb300._build --debug`): every
 * queue append, queue read and output store of the kernels checks its index
 * against the buffer's bound; a violation skips the access and is recorded
 * (no trap, so the context stays usable).  *sites receives the OR of the
 * violated sites' bits (bit k: site k; the sites are the classify queues
 * and output, the Miller-Rabin queues and outputs, the batched kernel's
 * shared queues and outputs, the range kernel's queue and output, the window
 * gather and the one-warp kernels' outputs), *violations their count, for the
 * current device, since the last reset (reset != 0 clears them after
 * reading).  *compiled (nullable) is 1 in the debug build and 0 in the
 * production build, where the checks are compiled out and both counts read 0.
 * Reads device memory: synchronise the work to be checked first. */
int isprime_debug_checks(int reset, uint32_t *sites, uint64_t *violations, int *compiled);

/* ---------------------------------------------------------------- misc */

const char *isprime_strerror(int status);
const char *isprime_last_error(void);
int isprime_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ISPRIME_H_ */
