// Handle layout shared by the C ABI translation units.
#pragma once
#include <memory>
#include <vector>

#include "core/core.h"

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
};

// called by dmrg_destroy before a handle goes away: every batch that uses it
// releases its merged plans now and answers DMRG_ERR_STATE from then on
void dmrg_internal_handle_gone(dmrg_handle* h);

// sets the calling thread's dmrg_last_error() message
void dmrg_internal_set_error(const char* msg);
