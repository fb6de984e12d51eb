// Exception barrier between the library's C++ host code and its C entry points.
//
// Host-side steps (the CSR analysis, the SELL-C-sigma and FP32 copies, the batch tables) use
// standard containers, which report a failed allocation by throwing.  No exception may cross
// an extern "C" boundary, so those steps run inside guarded(), which turns it into a status.
#pragma once

#include <new>
#include <stdexcept>

#include "pk.h"

namespace pk {

// Records why a host step failed (pk_last_error) and returns the status the caller sees:
// PK_ERR_OOM for a failed host allocation, PK_ERR_ARG for any other exception.
pk_status host_failure(bool oom) noexcept;

template <class F>
pk_status guarded(F&& f) noexcept {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return host_failure(true);
  } catch (const std::length_error&) {
    return host_failure(true);
  } catch (...) {
    return host_failure(false);
  }
}

}  // namespace pk
