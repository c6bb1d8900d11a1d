// Handle layout and the status mapping shared by the C ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dmrg_gb300.h"
#include "core/core.h"
#include "exec_errors.h"

struct dmrg_batch;

struct dmrg_handle {
  std::unique_ptr<dmrg::Exec> ex;
  std::unique_ptr<dmrg::Engine> eng;
  int L = 0;
  int device = 0;          // CUDA device current when the handle was created
  int left_loaded = 0;     // number of left sites loaded
  int right_loaded = -1;   // lowest right site loaded (L if none)
  bool any_loaded = false;
  std::vector<dmrg_batch*> batches;   // live batches that use this handle
  std::vector<double> t_user, v_user; // integrals in the caller's orbital numbering
  std::vector<double> log_rows;       // dmrg_sweep_log tables (library-owned)
  std::vector<int32_t> log_kept;
};

// called by dmrg_destroy before a handle goes away: every batch that uses it
// releases its merged plans now and answers DMRG_ERR_STATE from then on
void dmrg_internal_handle_gone(dmrg_handle* h);

// sets the calling thread's dmrg_last_error() message
void dmrg_internal_set_error(const char* msg);

inline dmrg_status dmrg_internal_fail(dmrg_status s, const std::string& m) {
  dmrg_internal_set_error(m.c_str());
  return s;
}

// Runs one entry point's body and maps every exception to its status, the same
// way for every entry point: CUDA runtime errors -> DMRG_ERR_CUDA, device or host
// allocation failures -> DMRG_ERR_OOM, bounded device waits that gave up ->
// DMRG_ERR_TIMEOUT, everything else the core throws (argument and call-order
// checks) -> DMRG_ERR_ARG.
template <class F>
dmrg_status dmrg_internal_guard(F&& f) {
  try {
    dmrg_internal_set_error("");
    return f();
  } catch (const dmrg::CudaError& e) {
    return dmrg_internal_fail(DMRG_ERR_CUDA, e.what());
  } catch (const dmrg::OomError& e) {
    return dmrg_internal_fail(DMRG_ERR_OOM, e.what());
  } catch (const dmrg::TimeoutError& e) {
    return dmrg_internal_fail(DMRG_ERR_TIMEOUT, e.what());
  } catch (const std::bad_alloc&) {
    return dmrg_internal_fail(DMRG_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return dmrg_internal_fail(DMRG_ERR_ARG, e.what());
  } catch (...) {
    return dmrg_internal_fail(DMRG_ERR_STATE, "unknown error");
  }
}

// Makes `device` the calling thread's current CUDA device for the guard's lifetime
// and restores the previous one afterwards (device < 0: no change), so that an
// entry point launches on its handle's device whatever device the caller has
// made current since the handle was created.
struct DmrgDeviceGuard {
  int prev = -1;
  explicit DmrgDeviceGuard(int device) {
    int cur = -1;
    if (device >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != device && cudaSetDevice(device) == cudaSuccess)
      prev = cur;
  }
  ~DmrgDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DmrgDeviceGuard(const DmrgDeviceGuard&) = delete;
  DmrgDeviceGuard& operator=(const DmrgDeviceGuard&) = delete;
};

// dmrg_internal_guard with the handle's device current during the call
template <class F>
dmrg_status dmrg_internal_guard_on(int device, F&& f) {
  return dmrg_internal_guard([&]() -> dmrg_status {
    DmrgDeviceGuard dg(device);
    return f();
  });
}

// Reads the executor's device error word (a stream synchronisation): 9 = the
// symmetric eigensolver did not converge (DMRG_ERR_NOCONV), any other nonzero
// value = a bounded tensor-core pipeline wait gave up (DMRG_ERR_TIMEOUT).
inline dmrg_status dmrg_internal_check_device(dmrg_handle* h) {
  const int code = h->eng->exec()->device_error();
  if (code == 9) return dmrg_internal_fail(DMRG_ERR_NOCONV, "the symmetric eigensolver did not converge");
  if (code) return dmrg_internal_fail(DMRG_ERR_TIMEOUT, "a tensor-core pipeline wait gave up; destroy the handle");
  return DMRG_OK;
}
