// Checks of the host runtime pieces that need no GPU (exits 0 when all hold):
//  - abi_guard: a failed host allocation -> QS_ENOMEM, any other exception ->
//    QS_EINVAL, each with a message naming the entry point; a normal return passes;
//  - parallel_for: every item runs exactly once; an exception from an item is
//    rethrown on the caller after all threads are done, and a later loop works;
//    host_threads() honours QS_HOST_THREADS.
// usage: host_runtime_check expected_threads.  Built against the library by
// test_host_runtime.py.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "abi_guard.h"
#include "host_par.h"
#include "qsim.h"

using namespace qs;

static int fails = 0;
static void check(bool ok, const char* what) {
  if (!ok) {
    std::fprintf(stderr, "FAILED: %s\n", what);
    ++fails;
  }
}

int main(int argc, char** argv) {
  if (argc != 2) return 2;
  // abi_guard
  qs_status s = abi_guard("entry_a", []() -> qs_status { throw std::bad_alloc(); });
  check(s == QS_ENOMEM, "bad_alloc -> QS_ENOMEM");
  check(std::string(qs_last_error()).find("entry_a") != std::string::npos, "message names the entry point");
  s = abi_guard("entry_b", []() -> qs_status { throw std::runtime_error("planner broke"); });
  check(s == QS_EINVAL, "runtime_error -> QS_EINVAL");
  check(std::string(qs_last_error()).find("planner broke") != std::string::npos, "message carries what()");
  s = abi_guard("entry_c", []() -> qs_status { throw 7; });
  check(s == QS_EINVAL, "non-std exception -> QS_EINVAL");
  s = abi_guard("entry_d", []() -> qs_status { return QS_EUNSUPPORTED; });
  check(s == QS_EUNSUPPORTED, "a returned status passes through");
  // parallel_for
  check(host_threads() == (size_t)std::atoi(argv[1]), "host_threads() as QS_HOST_THREADS sets it");
  const size_t n = 5000;
  std::vector<std::atomic<int>> hits(n);
  for (auto& h : hits) h.store(0);
  parallel_for(n, 1, [&](size_t i) { hits[i].fetch_add(1); });
  bool once = true;
  for (auto& h : hits) once = once && h.load() == 1;
  check(once, "every item exactly once");
  bool caught = false;
  try {
    parallel_for(n, 1, [&](size_t i) {
      if (i == 1234) throw std::runtime_error("item 1234");
    });
  } catch (const std::runtime_error& e) {
    caught = std::strcmp(e.what(), "item 1234") == 0;
  }
  check(caught, "an item's exception reaches the caller");
  std::atomic<size_t> sum{0};
  parallel_for(n, 1, [&](size_t i) { sum.fetch_add(i); });
  check(sum.load() == n * (n - 1) / 2, "a loop after a failed one runs every item");
  return fails == 0 ? 0 : 1;
}
