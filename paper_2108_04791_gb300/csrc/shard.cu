// shard.cu -- host-side planning of one job across devices.
//
// The result for each element depends on that element alone (Sec. 1), so a
// job splits across devices with no data exchange: contiguous ranges of a
// plain array, whole arrays of a batch balanced by size, and served requests
// sent to the least-loaded device.  Nothing here touches a device.
// The batch plan is longest-processing-time first (Graham, SIAM J. Appl.
// Math. 17, 1969): its largest shard is at most (4/3 - 1/(3k)) of the best
// possible for k shards, and at most the mean plus the largest array.
#include <algorithm>
#include <functional>
#include <numeric>
#include <queue>
#include <utility>
#include <vector>

#include "internal.h"

extern "C" {

int isprime_plan_contiguous(uint64_t n, uint32_t n_shards, uint64_t* begin) {
  if (n_shards == 0 || !begin) return ip::set_error(ISPRIME_EINVAL, "n_shards must be > 0 and begin non-NULL");
  const uint64_t q = n / n_shards, r = n % n_shards;
  begin[0] = 0;
  for (uint32_t s = 0; s < n_shards; ++s) begin[s + 1] = begin[s] + q + (s < r ? 1 : 0);
  return ISPRIME_OK;
}

int isprime_plan_batched(const uint64_t* sizes, size_t n_arrays, uint32_t n_shards,
                         uint32_t* owner, uint64_t* load) {
  if (n_shards == 0) return ip::set_error(ISPRIME_EINVAL, "n_shards must be > 0");
  if (n_arrays > 0 && (!sizes || !owner)) return ip::set_error(ISPRIME_EINVAL, "NULL sizes or owner");
  std::vector<size_t> order(n_arrays);
  std::iota(order.begin(), order.end(), (size_t)0);
  std::stable_sort(order.begin(), order.end(),
                   [sizes](size_t a, size_t b) { return sizes[a] > sizes[b]; });
  // min-heap of (total, shard): the least-loaded shard, lower index on ties
  using Entry = std::pair<uint64_t, uint32_t>;
  std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> heap;
  for (uint32_t s = 0; s < n_shards; ++s) heap.push({0, s});
  std::vector<uint64_t> total(n_shards, 0);
  for (size_t i : order) {
    const Entry e = heap.top();
    heap.pop();
    owner[i] = e.second;
    total[e.second] = e.first + sizes[i];
    heap.push({total[e.second], e.second});
  }
  if (load) std::copy(total.begin(), total.end(), load);
  return ISPRIME_OK;
}

int isprime_route_least_loaded(const uint64_t* outstanding, uint32_t n_devices, uint32_t* device) {
  if (n_devices == 0 || !outstanding || !device)
    return ip::set_error(ISPRIME_EINVAL, "n_devices must be > 0 and pointers non-NULL");
  uint32_t best = 0;
  for (uint32_t d = 1; d < n_devices; ++d)
    if (outstanding[d] < outstanding[best]) best = d;
  *device = best;
  return ISPRIME_OK;
}

}  // extern "C"
