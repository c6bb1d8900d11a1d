// Exception types the executors raise; the C ABI maps them to dmrg_status codes.
#pragma once
#include <stdexcept>
#include <string>

namespace dmrg {
struct CudaError : std::runtime_error {
  explicit CudaError(const std::string& m) : std::runtime_error(m) {}
};
struct OomError : std::runtime_error {
  explicit OomError(const std::string& m) : std::runtime_error(m) {}
};
struct TimeoutError : std::runtime_error {
  explicit TimeoutError(const std::string& m) : std::runtime_error(m) {}
};
}  // namespace dmrg
