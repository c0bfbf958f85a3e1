// Host-side parallel loop for the planners' independent per-item work.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <thread>
#include <vector>

namespace qs {

// Host threads the planners may use: the environment variable QS_HOST_THREADS
// (1 = the calling thread only) if set to a positive number, else the hardware
// threads; at most 8 either way.
inline size_t host_threads() {
  static const size_t cap = [] {
    const char* e = std::getenv("QS_HOST_THREADS");
    const long v = e ? std::strtol(e, nullptr, 10) : 0;
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t t = v > 0 ? (size_t)v : (size_t)(hw ? hw : 1);
    return std::min<size_t>(t, 8);
  }();
  return cap;
}

// Runs f(i) for every i in [0, n): on the calling thread and up to
// host_threads() - 1 more, one thread per min_items items at most, each claiming
// the next item from a shared counter.  The items must be independent (each f(i)
// writes only its own outputs), so the results do not depend on the thread
// count.  If a thread cannot be started, the threads already running (the caller
// among them) do the rest.  An exception from f stops the hand-out and, once every
// thread has finished, is rethrown on the calling thread (the first one caught).
template <class F>
void parallel_for(size_t n, size_t min_items, F&& f) {
  const size_t nt = std::min<size_t>(host_threads(), n / std::max<size_t>(min_items, 1));
  if (nt <= 1) {
    for (size_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<size_t> next{0};
  std::mutex mu;
  std::exception_ptr failure;
  auto work = [&]() {
    try {
      for (size_t i = next.fetch_add(1); i < n; i = next.fetch_add(1)) f(i);
    } catch (...) {
      next.store(n);
      std::lock_guard<std::mutex> g(mu);
      if (!failure) failure = std::current_exception();
    }
  };
  std::vector<std::thread> th;
  try {
    th.reserve(nt - 1);
    for (size_t t = 1; t < nt; ++t) th.emplace_back(work);
  } catch (...) {
    // fewer threads: the ones started (and the caller) take the rest
  }
  work();
  for (std::thread& t : th) t.join();
  if (failure) std::rethrow_exception(failure);
}

}  // namespace qs
