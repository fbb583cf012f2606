// Fork-join loop over [0, n) on host threads (planning and formatting of large batches).
#pragma once
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

namespace bs {

// calls body(i) for every i in [0, n); uses up to 16 threads when n >= min_parallel
// the host's hardware threads, read once (the query reads the system's CPU list)
inline unsigned host_threads() {
  static const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  return hw;
}

template <class F>
void parallel_for(int n, int min_parallel, F body) {
  const int threads = (n >= min_parallel) ? (int)std::min<unsigned>(16u, host_threads()) : 1;
  if (threads <= 1) {
    for (int i = 0; i < n; ++i) body(i);
    return;
  }
  std::atomic<int> next{0};
  constexpr int kChunk = 32;
  auto worker = [&] {
    for (;;) {
      const int lo = next.fetch_add(kChunk);
      if (lo >= n) return;
      const int hi = std::min(n, lo + kChunk);
      for (int i = lo; i < hi; ++i) body(i);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
}

}  // namespace bs
