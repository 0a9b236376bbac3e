// batched.cu -- many ragged arrays in one persistent launch.
//
// The array path of Sec. 6 applied to a batch: every element of every array
// goes through the same decision (sieve lookup, trial division, Miller-Rabin
// with the bases of Eq. 4), but the whole batch is one kernel launch instead
// of one pipeline per array.
//
// Work distribution: each array is cut into tiles of `tile` elements; a block
// takes the next tile from a global counter (one atomic per tile), so short
// and long arrays balance across the GPU.  Survivors of trial division stay
// in the block: they are appended to a shared-memory queue Q1, and whenever
// Q1 holds a full block of work all threads run the base-2 test on it (or
// the 32-bit test for values below 2^32); elements that pass go to a second
// shared queue Q2, and whenever Q2 holds a full block the six remaining
// bases run on it.  Warps therefore stay dense in both stages without any
// global queue, and a block drains its partial queues once no tiles remain.
// The counter reset and the launch are recorded once in a CUDA graph and
// replayed per call; the descriptors are read from device memory.
#include <string.h>

#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace ip {

// Arithmetic: Montgomery formulation 9 (32-bit words in PTX, the final
// correction on the multiply pipe) in both stages, 3-bit windows for the six
// bases (as the plain path's defaults), and trial division on two residues
// when the count is the default 15 primes.
constexpr int kImplB2 = 9, kImplRest = 9;
constexpr int kBatchWin = 3;

struct BatchParams {
  const BatchDesc* descs;
  const BatchHeader* hdr;
  uint32_t* tile_counter;
  const uint32_t* sieve;
  uint64_t sieve_limit;
  uint32_t ntd;
  uint64_t td_square;
  uint32_t tile;  // elements per tile
};

__device__ __forceinline__ void smem_push(bool want, uint64_t v, uint64_t addr, uint64_t* qv,
                                          uint64_t* qa, uint32_t* count, uint32_t cap) {
  const unsigned mask = __ballot_sync(0xFFFFFFFFu, want);
  if (mask == 0) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (want) {
    const uint32_t pos = base + __popc(mask & ((1u << lane) - 1u));
    if (IP_CHECK(pos < cap, kChkSmemQueue)) {
      qv[pos] = v;
      qa[pos] = addr;
    }
  }
}

// Shared-memory bytes of one block: Q1 (tile + block entries), Q2 (2 block
// entries), 16 bytes per entry, plus the window tables (2^kBatchWin per thread).
size_t batched_smem_bytes(uint32_t block, uint32_t tile) {
  return (size_t)(tile + block) * 16 + (size_t)(2 * block) * 16 +
         ((size_t)1 << kBatchWin) * block * 8;
}


template <int kNtd, bool kLucas>
__global__ void __launch_bounds__(256) batched_kernel(BatchParams p) {
  extern __shared__ __align__(16) uint64_t s_dyn[];
  __shared__ uint32_t s_n1, s_n2, s_tile, s_arr;
  const uint32_t B = blockDim.x, tid = threadIdx.x;
  const uint32_t q1cap = p.tile + B, q2cap = 2 * B;
  uint64_t* q1v = s_dyn;
  uint64_t* q1a = q1v + q1cap;
  uint64_t* q2v = q1a + q1cap;
  uint64_t* q2a = q2v + q2cap;
  uint64_t* tab = q2a + q2cap + tid;  // this thread's column, stride B
  const uint64_t total_tiles = p.hdr->total_tiles;
  const uint64_t n_arrays = p.hdr->n_arrays;
  if (tid == 0) {
    s_n1 = 0;
    s_n2 = 0;
  }
  __syncthreads();

  // Base-2 round on `cnt` entries taken from the top of Q1 (cnt <= B).
  auto round1 = [&](uint32_t n1, uint32_t cnt) {
    const bool mine = tid < cnt;
    uint64_t v = 0, a = 0;
    if (mine) {
      v = q1v[n1 - cnt + tid];
      a = q1a[n1 - cnt + tid];
    }
    __syncthreads();
    if (tid == 0) s_n1 = n1 - cnt;
    if (mine && v < (1ull << 32) && mr32_is_prime((uint32_t)v)) *reinterpret_cast<uint8_t*>(a) = 1;
    // base 2 with 4-bit windows (x 2^w mod n by a quotient estimate), every
    // lane of the warp taking part with the warp's largest nibble count
    // (lanes without a 64-bit value test a prime)
    const bool b2 = mine && v >= (1ull << 32);
    const uint64_t nb = b2 ? v : 0xFFFFFFFFFFFFFFC5ull;
    const int nib = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)base2_nibbles(nb));
    const bool pass = base2_passes_shift<kImplB2>(nb, nib) && b2;
    smem_push(pass, v, a, q2v, q2a, &s_n2, q2cap);
    __syncthreads();
  };
  // Six-base round on `cnt` entries from the top of Q2 (cnt <= B).
  auto round2 = [&](uint32_t n2, uint32_t cnt) {
    const bool mine = tid < cnt;
    uint64_t v = 0, a = 0;
    if (mine) {
      v = q2v[n2 - cnt + tid];
      a = q2a[n2 - cnt + tid];
    }
    __syncthreads();
    if (tid == 0) s_n2 = n2 - cnt;
    if (kLucas) {  // every thread of the block takes part (warp-synchronous test)
      if (lucas_warp<kImplRest>(mine ? v : 0xFFFFFFFFFFFFFFC5ull, mine)) *reinterpret_cast<uint8_t*>(a) = 1;
    } else if (rest64_is_prime_warp<kImplRest, kBatchWin>(mine ? v : 0xFFFFFFFFFFFFFFC5ull, mine, tab,
                                                          (int)B)) {
      *reinterpret_cast<uint8_t*>(a) = 1;
    }
    __syncthreads();
  };

  for (;;) {
    if (tid == 0) {
      const uint32_t t = atomicAdd(p.tile_counter, 1u);
      s_tile = t;
      if (t < total_tiles) {  // last array whose first tile is <= t
        uint64_t lo = 0, hi = n_arrays - 1;
        while (lo < hi) {
          const uint64_t mid = (lo + hi + 1) >> 1;
          if (p.descs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
        }
        s_arr = (uint32_t)lo;
      }
    }
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= total_tiles) break;
    const BatchDesc d = p.descs[s_arr];
    const uint64_t e0 = (uint64_t)(t - d.tile_begin) * p.tile;
    const uint64_t e1 = min(d.n, e0 + p.tile);
    for (uint64_t base = e0; base < e1; base += B) {
      const uint64_t e = base + tid;
      int dec = kComposite;
      uint64_t v = 0;
      if (e < e1) {
        v = d.in[e];
        dec = classify_value<kNtd, BatchParams, false, (kNtd == 15 ? 3 : 0)>(v, p);
        if (IP_CHECK(e < d.n, kChkBatchOut)) d.out[e] = (uint8_t)(dec == kPrime);
      }
      smem_push(dec == kMR64 || dec == kMR32, v, (uint64_t)(d.out + e), q1v, q1a, &s_n1, q1cap);
    }
    __syncthreads();
    uint32_t n1 = s_n1;
    while (n1 >= B) {
      round1(n1, B);
      uint32_t n2 = s_n2;
      while (n2 >= B) {
        round2(n2, B);
        n2 = s_n2;
      }
      n1 = s_n1;
    }
  }
  // No tiles left: drain the partial queues.
  const uint32_t n1 = s_n1;
  if (n1) round1(n1, n1);
  uint32_t n2 = s_n2;
  while (n2) {
    round2(n2, n2 < B ? n2 : B);
    n2 = s_n2;
  }
}

IP_CHECK_READER(check_read_batched)

using BatchLauncher = void (*)(const BatchParams&, unsigned, unsigned, size_t, cudaStream_t);

template <int kNtd, bool kLucas>
static void launch_batched_t(const BatchParams& p, unsigned grid, unsigned block, size_t smem,
                             cudaStream_t s) {
  batched_kernel<kNtd, kLucas><<<grid, block, smem, s>>>(p);
}

struct BatchVariant {
  BatchLauncher launch;
  const void* fn;
};

// Compiled trial-division counts; other counts use the runtime-count kernel.
template <bool kLucas>
static BatchVariant pick_ntd(uint32_t ntd) {
  switch (ntd) {
    case 15: return {launch_batched_t<15, kLucas>, reinterpret_cast<const void*>(&batched_kernel<15, kLucas>)};
    case 23: return {launch_batched_t<23, kLucas>, reinterpret_cast<const void*>(&batched_kernel<23, kLucas>)};
    default: return {launch_batched_t<-1, kLucas>, reinterpret_cast<const void*>(&batched_kernel<-1, kLucas>)};
  }
}

static BatchVariant pick_variant(uint32_t ntd, uint32_t rest_test) {
  return rest_test == 1 ? pick_ntd<true>(ntd) : pick_ntd<false>(ntd);
}

// Grid: every SM full of resident blocks (occupancy with this shared memory).
static int batched_grid(isprime_ctx* ctx, const BatchVariant& v, uint32_t block, size_t smem,
                        unsigned* grid) {
  IP_CUDA(cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  IP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v.fn, (int)block, smem));
  if (per_sm < 1) return set_error(ISPRIME_EINVAL, "batched kernel does not fit on an SM with this tuning");
  *grid = (unsigned)(ctx->sm_count * per_sm);
  return ISPRIME_OK;
}

void batch_state_free(BatchState* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->ev) cudaEventDestroy(b->ev);
  cudaFree(b->d_batch);
  if (b->h_batch) cudaFreeHost(b->h_batch);
  cudaFree(b->d_tile_counter);
  *b = BatchState{};
}

int batched_run(isprime_ctx* ctx, BatchState* bs, const isprime_array* arrays, size_t n_arrays,
                uint64_t warp_max, cudaStream_t s) {
  IP_NVTX("batched_run");
  const uint32_t block = ctx->tune.batch_block;
  uint64_t elems = 0;
  for (size_t i = 0; i < n_arrays; ++i) elems += arrays[i].n;
  if (elems == 0) return ISPRIME_OK;
  // A batch of at most warp_max elements in all takes the one-launch warp
  // path (lowest latency); its descriptors carry element prefix sums.
  const bool warp_form = elems <= warp_max && n_arrays < (1ull << 32);
  const uint32_t tile = warp_form ? 1u : 1u << ctx->tune.batch_tile_log2;
  // Host-side descriptors: tile prefix sums (arrays with n == 0 get no tiles).
  std::vector<BatchDesc> descs(n_arrays);
  uint64_t tiles = 0;
  for (size_t i = 0; i < n_arrays; ++i) {
    descs[i].in = arrays[i].d_in;
    descs[i].out = arrays[i].d_out;
    descs[i].n = arrays[i].n;
    descs[i].tile_begin = tiles;
    tiles += (arrays[i].n + tile - 1) / tile;
  }
  // The counter overshoots by one fetch per block: keep it far from wrapping.
  if (tiles >= (1ull << 31)) return set_error(ISPRIME_EINVAL, "batch has 2^31 tiles or more");
  const size_t bytes = sizeof(BatchHeader) + n_arrays * sizeof(BatchDesc);
  // Device and pinned staging buffers (grow as needed; growth invalidates the graph).
  if (bs->cap < bytes) {
    if (bs->ev_valid) IP_CUDA(cudaEventSynchronize(bs->ev));
    IP_CUDA(cudaStreamSynchronize(s));
    cudaFree(bs->d_batch);
    cudaFreeHost(bs->h_batch);
    bs->d_batch = nullptr;
    bs->h_batch = nullptr;
    bs->cap = 0;
    const size_t cap = std::max(bytes * 2, (size_t)4096);
    IP_CUDA(cudaMalloc(&bs->d_batch, cap));
    IP_CUDA(cudaMallocHost(&bs->h_batch, cap));
    bs->cap = cap;
    if (bs->exec) {
      cudaGraphExecDestroy(bs->exec);
      bs->exec = nullptr;
    }
  }
  if (!bs->ev) IP_CUDA(cudaEventCreateWithFlags(&bs->ev, cudaEventDisableTiming));
  if (!bs->d_tile_counter) IP_CUDA(cudaMalloc(&bs->d_tile_counter, 256));
  // The pinned buffer may still be read by the previous call's copy.
  if (bs->ev_valid) IP_CUDA(cudaEventSynchronize(bs->ev));
  BatchHeader h;
  h.n_arrays = n_arrays;
  h.total_tiles = tiles;
  memcpy(bs->h_batch, &h, sizeof h);
  memcpy(static_cast<char*>(bs->h_batch) + sizeof h, descs.data(), n_arrays * sizeof(BatchDesc));
  IP_CUDA(cudaMemcpyAsync(bs->d_batch, bs->h_batch, bytes, cudaMemcpyHostToDevice, s));
  IP_CUDA(cudaEventRecord(bs->ev, s));
  bs->ev_valid = true;
  if (warp_form) {
    const BatchDesc* d_descs =
        reinterpret_cast<const BatchDesc*>(static_cast<char*>(bs->d_batch) + sizeof(BatchHeader));
    int st = launch_small_batched(ctx, d_descs, (uint32_t)n_arrays, elems, s);
    if (st) return st;
    ctx->stats.elements += elems;
    return ISPRIME_OK;
  }

  // The graph: reset the tile counter, launch the persistent kernel.
  const BatchVariant v = pick_variant(ctx->tune.td_primes, ctx->tune.rest_test);
  const size_t smem = batched_smem_bytes(block, tile);
  // every parameter the recorded graph depends on, in disjoint bit fields
  const uint64_t key = (uint64_t)block | ((uint64_t)tile << 10) |
                       ((uint64_t)ctx->tune.td_primes << 26) |
                       ((uint64_t)ctx->tune.batch_blocks_per_sm << 32) |
                       ((uint64_t)ctx->tune.rest_test << 40) |
                       ((uint64_t)ctx->tune.sieve_cutover_log2 << 42);
  if (!bs->exec || bs->key != key) {
    if (bs->exec) {
      IP_CUDA(cudaStreamSynchronize(s));
      cudaGraphExecDestroy(bs->exec);
      bs->exec = nullptr;
    }
    unsigned grid = 0;
    int st = batched_grid(ctx, v, block, smem, &grid);
    if (st) return st;
    if (ctx->tune.batch_blocks_per_sm)
      grid = std::min(grid, (unsigned)(ctx->sm_count * ctx->tune.batch_blocks_per_sm));
    BatchParams p;
    p.descs = reinterpret_cast<const BatchDesc*>(static_cast<char*>(bs->d_batch) + sizeof(BatchHeader));
    p.hdr = reinterpret_cast<const BatchHeader*>(bs->d_batch);
    p.tile_counter = bs->d_tile_counter;
    p.sieve = ctx->d_sieve;
    p.sieve_limit = sieve_cut(ctx);
    p.ntd = ctx->tune.td_primes;
    p.td_square = td_square_for(ctx->tune.td_primes);
    p.tile = tile;
    cudaStream_t cs;
    IP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(bs->d_tile_counter, 0, sizeof(uint32_t), cs);
      v.launch(p, grid, block, smem, cs);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bs->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "capturing the batched graph");
    bs->key = key;
    bs->grid = grid;
  }
  TimedLaunch tl;
  int st = launch_begin(ctx, ISPRIME_K_BATCHED, s, &tl);
  if (st) return st;
  IP_CUDA(cudaGraphLaunch(bs->exec, s));
  if ((st = launch_end(ctx, s, &tl, "batched graph"))) return st;
  ctx->stats.elements += elems;
  return ISPRIME_OK;
}

}  // namespace ip
