// shard.cu -- host-side planning of one job across devices.
//
// The result for each element depends on that element alone (Sec. 1), so a
// job splits across devices with no data exchange: contiguous ranges of a
// plain array, whole arrays of a batch balanced by size, and served requests
// sent to the least-loaded device.  The planners touch no device;
// isprime_u64_host_multi runs a plain job on several devices by the
// contiguous plan, one host thread per device, with no exchange between them.
// The batch plan is longest-processing-time first (Graham, SIAM J. Appl.
// Math. 17, 1969): its largest shard is at most (4/3 - 1/(3k)) of the best
// possible for k shards, and at most the mean plus the largest array.
#include <algorithm>
#include <functional>
#include <numeric>
#include <queue>
#include <thread>
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

int isprime_u64_host_multi(const int* devices, uint32_t n_devices, const uint64_t* h_in,
                           uint8_t* h_out, size_t n) {
  IP_NVTX("isprime_u64_host_multi");
  if (n_devices == 0 || !devices) return ip::set_error(ISPRIME_EINVAL, "no devices given");
  if (n == 0) return ISPRIME_OK;
  if (!h_in || !h_out) return ip::set_error(ISPRIME_EINVAL, "NULL pointer with n > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) ndev = 0;
  for (uint32_t k = 0; k < n_devices; ++k)
    if (devices[k] < 0 || devices[k] >= ndev) return ip::set_error(ISPRIME_EINVAL, "device out of range");
  std::vector<uint64_t> begin(n_devices + 1);
  isprime_plan_contiguous(n, n_devices, begin.data());
  // contexts first (building a device's resident sieve is not thread-safe
  // with that device's other first uses), then one thread per shard
  std::vector<isprime_ctx*> ctx(n_devices, nullptr);
  for (uint32_t k = 0; k < n_devices; ++k) {
    int st = isprime_default_ctx(devices[k], &ctx[k]);
    if (st) return st;
  }
  std::vector<int> status(n_devices, ISPRIME_OK);
  std::vector<std::string> error(n_devices);
  std::vector<std::thread> threads;
  for (uint32_t k = 0; k < n_devices; ++k) {
    const uint64_t b = begin[k], len = begin[k + 1] - begin[k];
    if (len == 0) continue;
    threads.emplace_back([&, k, b, len] {
      status[k] = isprime_u64_host(ctx[k], h_in + b, h_out + b, len, nullptr);
      if (status[k]) error[k] = isprime_last_error();
    });
  }
  for (auto& t : threads) t.join();
  for (uint32_t k = 0; k < n_devices; ++k)
    if (status[k]) return ip::set_error(status[k], "device " + std::to_string(devices[k]) + ": " + error[k]);
  return ISPRIME_OK;
}

}  // extern "C"
