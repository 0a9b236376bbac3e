// autotune.cu -- picks launch and algorithm parameters by measurement.
//
// The paper chooses between its two array paths with linear fits measured on
// one machine (Sec. 6.2, Eqs. 7-8).  The GPU analogue here chooses the
// parameters that only affect speed (block sizes, grid occupancy, trial
// division count, Montgomery formulation, survivor-compaction threshold,
// sieve / Miller-Rabin cutover, batched tile size, and the array length up
// to which the one-launch path beats the queue path) by timing the caller's
// own sample on this GPU.  Search: coordinate descent (each
// parameter swept over its candidate values with the others held, two
// passes), every candidate timed as the best of three runs with CUDA events.
// Results are cached in a text file keyed by GPU name, SM count, CUDA
// runtime version and the sample size, so later processes skip the search.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace ip {

namespace {

using FieldPtr = uint32_t isprime_tuning::*;

struct Param {
  const char* name;
  FieldPtr field;
  std::vector<uint32_t> values;
  int modes;  // bit ISPRIME_TUNE_PLAIN and/or ISPRIME_TUNE_BATCHED
};

std::vector<Param> params() {
  const int P = 1 << ISPRIME_TUNE_PLAIN, B = 1 << ISPRIME_TUNE_BATCHED;
  return {
      {"td_primes", &isprime_tuning::td_primes, {7, 11, 15, 23, 31}, P | B},
      {"classify_block", &isprime_tuning::classify_block, {128, 256, 512}, P},
      {"mr_block", &isprime_tuning::mr_block, {64, 128, 256}, P},
      {"blocks_per_sm", &isprime_tuning::blocks_per_sm, {4, 8, 16, 32}, P},
      {"mont_impl", &isprime_tuning::mont_impl, {9, 6, 0, 5}, P},
      {"mont_impl_base2", &isprime_tuning::mont_impl_base2, {9, 6, 0, 5}, P},
      {"base2_window", &isprime_tuning::base2_window, {0, 1, 4}, P},
      {"compact_min", &isprime_tuning::compact_min, {33, 28, 24, 16}, P},
      {"td_fold", &isprime_tuning::td_fold, {0, 1, 2, 3}, P},
      {"base2_split", &isprime_tuning::base2_split, {0, 1}, P},
      {"base2_ilp", &isprime_tuning::base2_ilp, {1, 2}, P},
      {"rest_window", &isprime_tuning::rest_window, {4, 3}, P},
      {"rest_ilp", &isprime_tuning::rest_ilp, {1, 2}, P},
      {"base2_blocks_per_sm", &isprime_tuning::base2_blocks_per_sm, {4, 0, 6, 5}, P},
      {"pdl", &isprime_tuning::pdl, {0, 1}, P},
      {"td2_groups", &isprime_tuning::td2_groups, {0, 8, 12, 16, 24}, P},
      {"dual_stream", &isprime_tuning::dual_stream, {0, 1}, P},
      {"inplace_max_log2", &isprime_tuning::inplace_max_log2, {0, 17, 20, 24}, P},
      {"sieve_cutover_log2", &isprime_tuning::sieve_cutover_log2, {32, 28, 24, 20}, P | B},
      {"batch_block", &isprime_tuning::batch_block, {64, 128, 256}, B},
      {"batch_tile_log2", &isprime_tuning::batch_tile_log2, {8, 9, 10, 11, 12}, B},
  };
}

std::string cache_key(int device, size_t n, int mode) {
  cudaDeviceProp prop;
  int rt = 0;
  cudaGetDeviceProperties(&prop, device);
  cudaRuntimeGetVersion(&rt);
  char buf[512];
  snprintf(buf, sizeof buf, "%s|sm%d|cudart%d|n%zu|mode%d", prop.name, prop.multiProcessorCount, rt, n,
           mode);
  std::string k(buf);
  for (auto& c : k)
    if (c == ' ' || c == '\t' || c == '=') c = '_';
  return k;
}

const char* kFields[] = {"classify_block", "mr_block", "blocks_per_sm", "td_primes", "chunk_log2",
                         "mont_impl", "mont_impl_base2", "batch_block", "batch_tile_log2",
                         "batch_blocks_per_sm", "base2_window", "rest_test", "small_max",
                         "compact_min", "sieve_cutover_log2", "serve_short_max", "td_fold",
                         "base2_split", "base2_ilp", "rest_window", "window_ratio16",
                         "base2_blocks_per_sm", "pdl", "td2_groups", "dual_stream", "host_chunk_log2", "inplace_max_log2",
                         "serve_long_log2", "rest_ilp"};
FieldPtr kFieldPtr[] = {
    &isprime_tuning::classify_block, &isprime_tuning::mr_block, &isprime_tuning::blocks_per_sm,
    &isprime_tuning::td_primes, &isprime_tuning::chunk_log2, &isprime_tuning::mont_impl,
    &isprime_tuning::mont_impl_base2, &isprime_tuning::batch_block,
    &isprime_tuning::batch_tile_log2, &isprime_tuning::batch_blocks_per_sm,
    &isprime_tuning::base2_window, &isprime_tuning::rest_test, &isprime_tuning::small_max,
    &isprime_tuning::compact_min, &isprime_tuning::sieve_cutover_log2,
    &isprime_tuning::serve_short_max, &isprime_tuning::td_fold, &isprime_tuning::base2_split,
    &isprime_tuning::base2_ilp, &isprime_tuning::rest_window, &isprime_tuning::window_ratio16,
    &isprime_tuning::base2_blocks_per_sm, &isprime_tuning::pdl, &isprime_tuning::td2_groups,
    &isprime_tuning::dual_stream, &isprime_tuning::host_chunk_log2,
    &isprime_tuning::inplace_max_log2, &isprime_tuning::serve_long_log2,
    &isprime_tuning::rest_ilp};
constexpr int kNumFields = 29;

std::string format_tuning(const isprime_tuning& t) {
  std::string s;
  for (int i = 0; i < kNumFields; ++i) {
    s += kFields[i];
    s += "=";
    s += std::to_string(t.*kFieldPtr[i]);
    s += i + 1 < kNumFields ? "," : "";
  }
  return s;
}

bool parse_tuning(const std::string& s, isprime_tuning* t) {
  size_t pos = 0;
  int got = 0;
  while (pos < s.size()) {
    size_t comma = s.find(',', pos);
    if (comma == std::string::npos) comma = s.size();
    const std::string kv = s.substr(pos, comma - pos);
    const size_t eq = kv.find('=');
    if (eq != std::string::npos) {
      const std::string k = kv.substr(0, eq);
      const unsigned long v = strtoul(kv.c_str() + eq + 1, nullptr, 10);
      for (int i = 0; i < kNumFields; ++i)
        if (k == kFields[i]) {
          t->*kFieldPtr[i] = (uint32_t)v;
          ++got;
        }
    }
    pos = comma + 1;
  }
  return got == kNumFields;
}

bool cache_lookup(const char* path, const std::string& key, isprime_tuning* t) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[2048];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    std::string l(line);
    while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
    const size_t sp = l.find(' ');
    if (sp == std::string::npos || l.compare(0, sp, key) != 0) continue;
    isprime_tuning cand = *t;
    if (parse_tuning(l.substr(sp + 1), &cand)) {
      *t = cand;
      found = true;  // the last matching line wins
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const isprime_tuning& t) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %s\n", key.c_str(), format_tuning(t).c_str());
  fclose(f);
}

}  // namespace

// Times one configuration: best of `reps` runs of the plain or batched path.
static int time_config(isprime_ctx* ctx, const uint64_t* d_in, uint8_t* d_out, size_t n,
                       const std::vector<isprime_array>& batch, bool batched, cudaStream_t s,
                       cudaEvent_t e0, cudaEvent_t e1, int reps, float* best_ms) {
  *best_ms = 1e30f;
  for (int r = 0; r < reps + 1; ++r) {  // first run warms up (and records the graph)
    IP_CUDA(cudaEventRecord(e0, s));
    int st = batched ? isprime_u64_batched(ctx, batch.data(), batch.size(), (isprime_stream)s)
                     : isprime_u64_ctx(ctx, d_in, d_out, n, (isprime_stream)s);
    if (st) return st;
    IP_CUDA(cudaEventRecord(e1, s));
    IP_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    IP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (r > 0) *best_ms = std::min(*best_ms, ms);
  }
  return ISPRIME_OK;
}

int autotune(isprime_ctx* ctx, const uint64_t* d_sample, uint8_t* d_out, size_t n, int mode,
             const char* cache_path, isprime_tuning* result) {
  const std::string key = cache_key(ctx->device, n, mode);
  isprime_tuning t = ctx->tune;
  if (cache_lookup(cache_path, key, &t)) {
    int st = isprime_ctx_set_tuning(ctx, &t);
    if (st) return st;
    if (result) *result = t;
    return ISPRIME_OK;
  }
  const bool batched = mode == ISPRIME_TUNE_BATCHED;
  // The batched sample: the sample cut into ragged pieces of growing length.
  std::vector<isprime_array> batch;
  for (size_t off = 0, len = 1; off < n; off += len, len = std::min(len * 3 + 1, (size_t)1 << 20)) {
    const size_t m = std::min(len, n - off);
    batch.push_back({d_sample + off, d_out + off, m});
  }
  cudaStream_t s;
  IP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  IP_CUDA(cudaEventCreate(&e0));
  IP_CUDA(cudaEventCreate(&e1));
  int st = ISPRIME_OK;
  float best = 0;
  st = time_config(ctx, d_sample, d_out, n, batch, batched, s, e0, e1, 3, &best);
  for (int pass = 0; pass < 2 && !st; ++pass) {
    for (const Param& p : params()) {
      if (!(p.modes & (1 << mode))) continue;
      for (uint32_t v : p.values) {
        isprime_tuning cand = t;
        if (cand.*(p.field) == v) continue;
        cand.*(p.field) = v;
        if (isprime_ctx_set_tuning(ctx, &cand) != ISPRIME_OK) continue;
        float ms = 0;
        st = time_config(ctx, d_sample, d_out, n, batch, batched, s, e0, e1, 3, &ms);
        if (st) break;
        if (ms < best * 0.99f) {  // keep a candidate only for a clear gain
          best = ms;
          t = cand;
        }
        isprime_ctx_set_tuning(ctx, &t);
      }
      if (st) break;
    }
  }
  // Array-level path choice (what Sec. 6.2's Eqs. 7-8 decide between the
  // paper's two array paths, here measured rather than fitted): the one-
  // launch warp-per-element path against the queue path on prefixes of the
  // sample of 64 ... 2^20 elements; small_max becomes the largest length at
  // which the warp path is still faster.
  if (!st && !batched) {
    uint32_t best_small = 0;
    for (size_t m = 64; m <= std::min(n, (size_t)1 << 20) && !st; m *= 2) {
      float ms_warp = 0, ms_queue = 0;
      isprime_tuning cand = t;
      cand.small_max = 1u << 20;
      if ((st = isprime_ctx_set_tuning(ctx, &cand))) break;
      if ((st = time_config(ctx, d_sample, d_out, m, batch, false, s, e0, e1, 10, &ms_warp))) break;
      cand.small_max = 0;
      if ((st = isprime_ctx_set_tuning(ctx, &cand))) break;
      if ((st = time_config(ctx, d_sample, d_out, m, batch, false, s, e0, e1, 10, &ms_queue))) break;
      if (ms_warp >= ms_queue) break;
      best_small = (uint32_t)m;
    }
    t.small_max = best_small;
  }
  // The window path (window.cu): its crossover on this GPU near the sample's
  // largest value; installed when the sample itself is a window the fitted
  // rule takes (its values dense in [min, max] above the sieve limit).
  if (!st && !batched) {
    isprime_ctx_set_tuning(ctx, &t);
    uint64_t lo = 0, hi = 0;
    uint32_t r16 = 0;
    st = array_minmax(ctx, d_sample, n, s, &lo, &hi);
    if (!st) st = window_fit(ctx, hi, n, s, &r16);
    const unsigned __int128 w = (unsigned __int128)(hi - lo) + 1;
    if (!st && r16 && n >= ((size_t)1 << 16) && hi >= sieve_cut(ctx) &&
        w <= ((unsigned __int128)1 << 30) && w * 16 <= (unsigned __int128)n * r16)
      t.window_ratio16 = r16;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (st) return st;
  isprime_ctx_set_tuning(ctx, &t);
  cache_store(cache_path, key, t);
  if (result) *result = t;
  return ISPRIME_OK;
}

}  // namespace ip

extern "C" int isprime_autotune(isprime_ctx* ctx, const uint64_t* d_sample, uint8_t* d_scratch_out,
                                size_t n, int mode, const char* cache_path, isprime_tuning* out) {
  IP_NVTX("isprime_autotune");
  if (!ctx || !d_sample || !d_scratch_out || n == 0)
    return ip::set_error(ISPRIME_EINVAL, "autotune needs a context and a non-empty device sample");
  if (mode != ISPRIME_TUNE_PLAIN && mode != ISPRIME_TUNE_BATCHED)
    return ip::set_error(ISPRIME_EINVAL, "mode must be ISPRIME_TUNE_PLAIN or ISPRIME_TUNE_BATCHED");
  return ip::autotune(ctx, d_sample, d_scratch_out, n, mode, cache_path, out);
}

extern "C" int isprime_tuning_format(const isprime_tuning* t, char* buf, size_t cap) {
  if (!t || !buf || cap == 0) return ip::set_error(ISPRIME_EINVAL, "NULL argument");
  const std::string s = ip::format_tuning(*t);
  snprintf(buf, cap, "%s", s.c_str());
  return s.size() < cap ? ISPRIME_OK : ip::set_error(ISPRIME_EINVAL, "buffer too small");
}
