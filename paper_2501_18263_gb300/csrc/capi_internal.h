// Handle layout shared by the C ABI translation units.
#pragma once
#include <memory>

#include "core/core.h"

struct dmrg_handle {
  std::unique_ptr<dmrg::Exec> ex;
  std::unique_ptr<dmrg::Engine> eng;
  int L = 0;
  int device = 0;          // CUDA device current when the handle was created
  int left_loaded = 0;     // number of left sites loaded
  int right_loaded = -1;   // lowest right site loaded (L if none)
  bool any_loaded = false;
};

// sets the calling thread's dmrg_last_error() message
void dmrg_internal_set_error(const char* msg);
