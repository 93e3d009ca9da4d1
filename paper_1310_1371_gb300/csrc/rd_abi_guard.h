// The C boundary: no C++ exception leaves an extern "C" entry point.
//
// Entry points that can allocate host memory (std::string messages, std::vector
// tables, a server's request copies) or start a thread run their body through
// rd_guard.  An exception ends the call with a status: RD_E_NOMEM for a failed
// host allocation, RD_E_HOST for any other C++ failure (a thread that could
// not start).  The message goes to the entry point's last-error string when
// that assignment itself succeeds.  What the body had acquired is released by
// its own owners (the callers of rd_guard hold contexts and servers in scope
// guards until they hand them out).
#pragma once

#include <exception>
#include <new>
#include <string>

#include "rd.h"

namespace rd_abi {

inline void note(std::string* err, const char* m) noexcept {
  if (!err) return;
  try {
    *err = m;
  } catch (...) {
  }
}

// Entry points that return an rd_status.
template <typename Body>
inline rd_status guard(std::string* err, Body&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    note(err, "host memory allocation failed");
    return RD_E_NOMEM;
  } catch (const std::exception& e) {
    note(err, e.what());
    return RD_E_HOST;
  } catch (...) {
    note(err, "unknown C++ exception");
    return RD_E_HOST;
  }
}

// Entry points that return a count, or -1 on failure.
template <typename Body>
inline int guard_count(std::string* err, Body&& body) noexcept {
  try {
    return body();
  } catch (const std::exception& e) {
    note(err, e.what());
    return -1;
  } catch (...) {
    note(err, "unknown C++ exception");
    return -1;
  }
}

}  // namespace rd_abi
