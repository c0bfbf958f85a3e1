// Host-side parallel loop for the planners' independent per-item work.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <thread>
#include <vector>

namespace qs {

// Runs f(i) for every i in [0, n): on the calling thread and up to 7 more, one
// thread per min_items items at most, each claiming the next item from a shared
// counter.  The items must be independent (each f(i) writes only its own
// outputs), so the results do not depend on the thread count.  If a thread
// cannot be started, the threads already running (the caller among them) do the
// rest.
template <class F>
void parallel_for(size_t n, size_t min_items, F&& f) {
  const unsigned hw = std::thread::hardware_concurrency();
  const size_t nt = std::min<size_t>({(size_t)(hw ? hw : 1), (size_t)8, n / std::max<size_t>(min_items, 1)});
  if (nt <= 1) {
    for (size_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (size_t i = next.fetch_add(1); i < n; i = next.fetch_add(1)) f(i);
  };
  std::vector<std::thread> th;
  th.reserve(nt - 1);
  for (size_t t = 1; t < nt; ++t) {
    try {
      th.emplace_back(work);
    } catch (...) {
      break;
    }
  }
  work();
  for (std::thread& t : th) t.join();
}

}  // namespace qs
