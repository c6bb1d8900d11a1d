// dmrg_sigma_host_noalloc: the host-buffer sigma step without any device
// allocation.  dmrg_sigma_host stages psi and sigma in a device buffer that it
// allocates on every call; this variant stages them in a file-scope device
// array instead, for callers that must not allocate device memory while they
// run: a service that sized its device memory once at start-up and may not
// grow it afterwards, or a caller whose allocator is owned by someone else
// (a framework's memory pool, a fixed arena) and must not be entered from here.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../capi_internal.h"

namespace {

// Staging for one call: psi in [0, kMaxPsi), sigma in [kMaxPsi, 2 kMaxPsi).
// 2 x 2^21 doubles = 32 MiB, held by every device that loads the library.
constexpr int64_t kMaxPsi = int64_t(1) << 21;
__device__ __align__(256) double g_staging[2 * kMaxPsi];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

dmrg_status fail(dmrg_status s, const std::string& m) { return dmrg_internal_fail(s, m); }

}  // namespace

extern "C" dmrg_status dmrg_sigma_host_noalloc(dmrg_handle* h, int32_t bond, const double* psi_host,
                                               double* sigma_host) {
  return dmrg_internal_guard([&]() -> dmrg_status {
    if (!h || !psi_host || !sigma_host) return fail(DMRG_ERR_ARG, "null argument");
    if (h->eng->bond() != bond)
      return fail(DMRG_ERR_ARG, "bond not prepared: call dmrg_prepare for this bond first");
    const int64_t n = h->eng->psi_size();
    if (n > kMaxPsi)
      return fail(DMRG_ERR_ARG, "psi_size " + std::to_string(n) + " exceeds the allocation-free limit of " +
                                    std::to_string(kMaxPsi) + " doubles; use dmrg_sigma_host");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(DMRG_ERR_CUDA, "cudaGetDevice failed");
    if (cur != h->device) return fail(DMRG_ERR_ARG, "the handle's device is not the current device");
    if (cur < 0 || cur >= kMaxDevices) return fail(DMRG_ERR_ARG, "device ordinal out of range");
    double* base = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_mu);
      if (!g_addr[cur]) {
        // once per device, with that device current: device address of the array
        void* p = nullptr;
        cudaError_t rc = cudaGetSymbolAddress(&p, g_staging);
        if (rc != cudaSuccess)
          return fail(DMRG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(rc));
        g_addr[cur] = static_cast<double*>(p);
      }
      base = g_addr[cur];
    }
    dmrg::Exec* ex = h->eng->exec();
    ex->h2d_direct(base, psi_host, size_t(n) * sizeof(double));
    // replays the bond's CUDA graph if one was captured earlier; never captures one
    // here (instantiating a graph may allocate)
    h->eng->sigma_precision(base, base + kMaxPsi, h->eng->problem().precision, false);
    ex->d2h(sigma_host, base + kMaxPsi, size_t(n) * sizeof(double));
    // the same device status mapping as every other entry point
    return dmrg_internal_check_device(h);
  });
}
