// Exceptions stop at the C ABI.
#pragma once

#include <exception>
#include <new>

#include "internal.h"

namespace qs {

// Runs the body of a C-ABI entry point.  A C++ exception from the host code
// beneath it (an allocation in a planner, a container, a thread start) must not
// cross the C boundary: it becomes a status with a message (qs_last_error) --
// QS_ENOMEM for a failed host allocation, QS_EINVAL for anything else.
template <class F>
qs_status abi_guard(const char* fn, F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    set_error("%s: out of host memory", fn);
    return QS_ENOMEM;
  } catch (const std::exception& e) {
    set_error("%s: %s", fn, e.what());
    return QS_EINVAL;
  } catch (...) {
    set_error("%s: unexpected failure", fn);
    return QS_EINVAL;
  }
}

}  // namespace qs
