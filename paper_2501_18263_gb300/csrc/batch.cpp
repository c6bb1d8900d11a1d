// Batched form of the sigma step: many independent problems (handles prepared
// at their bonds) share one grouped tensor-core launch per stage, and the whole
// step can be captured once into a CUDA graph and replayed.
//
// The split-BF16 sigma of one problem is: psi -> split planes, local term H_L',
// stage 1 (X_nu = O_L psi), stage 2 (sigma = sum_nu X_nu O_R^T, split-K parts),
// fixed-order reduction of the parts, double-float -> FP64.  The two stages and
// the local term are grouped GEMMs over a tile list; their plans hold absolute
// device addresses, so the plans of several problems concatenate into one list
// whose tiles, sorted together by work, keep every SM busy even when each
// problem alone is too small to fill the GPU.  Each output tile is computed
// exactly as in the single-problem launch, so the batched sigma equals the
// per-problem sigma bit for bit.
#include <cuda_runtime.h>

#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dmrg_gb300.h"
#include "capi_internal.h"
#include "exec_errors.h"

struct dmrg_batch {
  std::vector<dmrg_handle*> h;
  std::vector<int> bond;
  std::vector<uint64_t> gen;
  dmrg::Exec* owner = nullptr;   // executor of the first handle: holds the merged plans
  int device = -1;               // the handles' CUDA device (made current by every batch call)
  cudaStream_t st = nullptr;
  int plan_hl = -1, plan1 = -1, plan2 = -1;
  // captured graph and the buffers it was captured with
  std::vector<const double*> g_psi;
  std::vector<double*> g_sig;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool dead = false;   // one of its handles was destroyed: plans released
  int order[3] = {0, 0, 0};                  // chosen tile order: local term, stage 1, stage 2
  int width[3] = {128, 128, 128};            // chosen tile width (MMA N) of the same launches
  float ms[3][6] = {};                       // measured ms per candidate: [2 order + (width == 64)]
};

namespace {

dmrg_status fail(dmrg_status s, const std::string& m) { return dmrg_internal_fail(s, m); }

template <class F>
dmrg_status guard(F&& f) {
  return dmrg_internal_guard(std::forward<F>(f));
}

// one plan made of the given plans of several executors: problems, segments and
// gathered-row tables concatenated, indices offset
struct Merged {
  std::vector<dmrg::MixProb> P;
  std::vector<dmrg::MixSeg> S;
  std::vector<int64_t> bcol, ccol;
  std::vector<float> acol;
};

Merged merge(const std::vector<std::pair<dmrg::Exec*, int>>& parts) {
  Merged m;
  auto& P = m.P;
  auto& S = m.S;
  auto& bcol = m.bcol;
  auto& ccol = m.ccol;
  auto& acol = m.acol;
  for (const auto& pr : parts) {
    if (pr.second < 0) continue;
    const dmrg::Exec::MixPlanHost& H = pr.first->mix_plan_host(pr.second);
    // a gathered 8-row unit has two bcol entries and eight ccol / acol entries
    if (H.bcol.size() * 4 != H.ccol.size() || H.acol.size() != H.ccol.size())
      throw std::runtime_error("batch: gathered-row tables of a plan are inconsistent");
    const int so = int(S.size());
    const int64_t co = int64_t(ccol.size());
    for (dmrg::MixProb q : H.p) {
      q.s0 += so;
      q.s1 += so;
      if (q.mode == 3) q.cm0 += co;
      P.push_back(q);
    }
    S.insert(S.end(), H.s.begin(), H.s.end());
    bcol.insert(bcol.end(), H.bcol.begin(), H.bcol.end());
    ccol.insert(ccol.end(), H.ccol.begin(), H.ccol.end());
    acol.insert(acol.end(), H.acol.begin(), H.acol.end());
  }
  return m;
}

// Autotuner of the merged launch's tile schedule and tile shape: every candidate
// (three orders x tile widths 128 and 64, or the one width the caller fixed) is
// built and timed on the GPU (CUDA events, one warm-up run), the fastest is kept.
// All candidates compute every output element with the same products in the same
// order, so the choice changes only the time.  Running a plan here is harmless:
// it writes only the handles' own intermediate buffers, which every sigma step
// rewrites before reading.  ms_out[2 order + (width == 64)] receives the times.
int build_tuned(dmrg::Exec* owner, const Merged& m, bool tune, int fixed_width, int* order_out, int* width_out,
                float* ms_out) {
  if (m.P.empty()) return -1;
  const int w0 = fixed_width > 0 ? fixed_width : 128;
  if (!tune) {
    *order_out = 0;
    *width_out = w0;
    return owner->mix_plan_ordered(m.P, m.S, m.bcol, m.ccol, m.acol, 0, w0);
  }
  std::vector<int> widths{w0};
  if (fixed_width <= 0) widths.push_back(64);
  int best = -1;
  float best_ms = 0.f;
  for (int order = 0; order < 3; ++order)
    for (int w : widths) {
      const int id = owner->mix_plan_ordered(m.P, m.S, m.bcol, m.ccol, m.acol, order, w);
      const float ms = owner->mix_time(id, 2);
      ms_out[2 * order + (w == 64 ? 1 : 0)] = ms;
      if (best < 0 || ms < best_ms) {
        if (best >= 0) owner->mix_plan_free(best);
        best = id;
        best_ms = ms;
        *order_out = order;
        *width_out = w;
      } else {
        owner->mix_plan_free(id);
      }
    }
  return best;
}

void free_graph(dmrg_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->g_psi.clear();
  b->g_sig.clear();
}

// release the merged plans (while the owner executor exists) and detach the
// batch from its handles; afterwards the batch holds nothing but its own memory
void retire(dmrg_batch* b) {
  if (b->dead) return;
  free_graph(b);
  for (int id : {b->plan_hl, b->plan1, b->plan2})
    if (id >= 0) b->owner->mix_plan_free(id);
  b->plan_hl = b->plan1 = b->plan2 = -1;
  b->owner->sync();
  for (dmrg_handle* h : b->h) {
    auto& v = h->batches;
    for (size_t i = 0; i < v.size(); ++i)
      if (v[i] == b) {
        v.erase(v.begin() + long(i));
        break;
      }
  }
  b->dead = true;
}

// the batched step, issued on the shared stream (no allocation, no host wait)
void issue(dmrg_batch* b, const double* const* psi, double* const* sig) {
  for (size_t i = 0; i < b->h.size(); ++i) b->h[i]->eng->batch_prologue(psi[i]);
  if (b->plan_hl >= 0) b->owner->mix_run(b->plan_hl);
  if (b->plan1 >= 0) b->owner->mix_run(b->plan1);
  for (size_t i = 0; i < b->h.size(); ++i) b->h[i]->eng->batch_zero_parts();
  if (b->plan2 >= 0) b->owner->mix_run(b->plan2);
  for (size_t i = 0; i < b->h.size(); ++i) b->h[i]->eng->batch_epilogue(sig[i]);
}

}  // namespace

extern "C" {

dmrg_status dmrg_batch_create(int32_t n, dmrg_handle* const* handles, const int32_t* bonds, dmrg_batch** out) {
  return dmrg_batch_create_ex(n, handles, bonds, 0, out);
}

dmrg_status dmrg_batch_create_ex(int32_t n, dmrg_handle* const* handles, const int32_t* bonds, int32_t tile_width,
                                 dmrg_batch** out) {
  const int dev = (n > 0 && handles && handles[0]) ? handles[0]->device : -1;
  return dmrg_internal_guard_on(dev, [&]() -> dmrg_status {
    if (!out || n <= 0 || !handles || !bonds) return fail(DMRG_ERR_ARG, "bad arguments");
    if (tile_width != 0 && tile_width != 64 && tile_width != 128)
      return fail(DMRG_ERR_ARG, "tile_width must be 0 (tuned), 64 or 128");
    *out = nullptr;
    auto b = std::make_unique<dmrg_batch>();
    for (int i = 0; i < n; ++i) {
      dmrg_handle* h = handles[i];
      if (!h) return fail(DMRG_ERR_ARG, "null handle");
      for (int j = 0; j < i; ++j)
        if (handles[j] == h) return fail(DMRG_ERR_ARG, "a handle appears twice in the batch");
      if (h->eng->problem().precision != DMRG_PREC_MIXED_BF16)
        return fail(DMRG_ERR_ARG, "batched sigma needs handles created with DMRG_PREC_MIXED_BF16");
      if (h->eng->bond() != bonds[i]) return fail(DMRG_ERR_ARG, "handle " + std::to_string(i) + " is not prepared at its bond");
      if (!h->eng->batchable())
        return fail(DMRG_ERR_ARG, "handle " + std::to_string(i) + " splits its terms into several chunks (memory cap)");
      if (h->device != handles[0]->device) return fail(DMRG_ERR_ARG, "handles on different devices");
      if (h->eng->exec()->stream() != handles[0]->eng->exec()->stream())
        return fail(DMRG_ERR_ARG, "handles must share one CUDA stream");
      b->h.push_back(h);
      b->bond.push_back(bonds[i]);
      b->gen.push_back(h->eng->plan_generation());
    }
    b->owner = handles[0]->eng->exec();
    b->device = handles[0]->device;
    b->st = static_cast<cudaStream_t>(b->owner->stream());
    std::vector<std::pair<dmrg::Exec*, int>> hl, p1, p2;
    for (dmrg_handle* h : b->h) {
      hl.push_back({h->eng->exec(), h->eng->mix_plan_hl()});
      p1.push_back({h->eng->exec(), h->eng->mix_plan1()});
      p2.push_back({h->eng->exec(), h->eng->mix_plan2()});
    }
    const bool tune = !b->owner->profiling();   // timing runs would pollute the caller's kernel profile
    try {
      b->plan_hl = build_tuned(b->owner, merge(hl), false, tile_width, &b->order[0], &b->width[0], b->ms[0]);
      b->plan1 = build_tuned(b->owner, merge(p1), tune, tile_width, &b->order[1], &b->width[1], b->ms[1]);
      b->plan2 = build_tuned(b->owner, merge(p2), tune, tile_width, &b->order[2], &b->width[2], b->ms[2]);
      b->owner->sync();
    } catch (...) {
      for (int id : {b->plan_hl, b->plan1, b->plan2})
        if (id >= 0) b->owner->mix_plan_free(id);
      throw;
    }
    for (dmrg_handle* h : b->h) h->batches.push_back(b.get());
    *out = b.release();
    return DMRG_OK;
  });
}

dmrg_status dmrg_batch_sigma(dmrg_batch* b, const double* const* psi_dev, double* const* sigma_dev,
                             int32_t use_graph) {
  return dmrg_internal_guard_on(b ? b->device : -1, [&]() -> dmrg_status {
    if (!b || !psi_dev || !sigma_dev) return fail(DMRG_ERR_ARG, "null argument");
    if (b->dead) return fail(DMRG_ERR_STATE, "a handle of the batch was destroyed; destroy the batch");
    const size_t n = b->h.size();
    for (size_t i = 0; i < n; ++i) {
      if (!psi_dev[i] || !sigma_dev[i]) return fail(DMRG_ERR_ARG, "null buffer");
      if (b->h[i]->eng->bond() != b->bond[i] || b->h[i]->eng->plan_generation() != b->gen[i])
        return fail(DMRG_ERR_STATE, "a handle of the batch was prepared again; destroy and recreate the batch");
    }
    if (use_graph) {
      if (b->st == nullptr) return fail(DMRG_ERR_ARG, "the graph form needs handles on a created (non-default) stream");
      for (dmrg_handle* h : b->h)
        if (h->eng->exec()->profiling()) return fail(DMRG_ERR_ARG, "kernel timing is on; the graph form cannot capture it");
      bool same = b->gexec != nullptr;
      for (size_t i = 0; same && i < n; ++i) same = b->g_psi[i] == psi_dev[i] && b->g_sig[i] == sigma_dev[i];
      if (!same) {
        free_graph(b);
        cudaError_t rc = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
        if (rc != cudaSuccess) return fail(DMRG_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(rc));
        try {
          issue(b, psi_dev, sigma_dev);
        } catch (...) {
          cudaGraph_t g = nullptr;
          cudaStreamEndCapture(b->st, &g);
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          throw;
        }
        rc = cudaStreamEndCapture(b->st, &b->graph);
        if (rc != cudaSuccess) {
          b->graph = nullptr;
          return fail(DMRG_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(rc));
        }
        rc = cudaGraphInstantiate(&b->gexec, b->graph, 0);
        if (rc != cudaSuccess) {
          b->gexec = nullptr;
          free_graph(b);
          return fail(DMRG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(rc));
        }
        b->g_psi.assign(psi_dev, psi_dev + n);
        b->g_sig.assign(sigma_dev, sigma_dev + n);
      }
      cudaError_t rc = cudaGraphLaunch(b->gexec, b->st);
      if (rc != cudaSuccess) return fail(DMRG_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(rc));
    } else {
      issue(b, psi_dev, sigma_dev);
    }
    b->owner->sync();
    if (b->owner->device_error()) return fail(DMRG_ERR_TIMEOUT, "a tensor-core pipeline wait gave up; destroy the handles");
    return DMRG_OK;
  });
}

dmrg_status dmrg_batch_schedule(dmrg_batch* b, int32_t* order3, float* ms9) {
  return guard([&]() -> dmrg_status {
    if (!b || !order3) return fail(DMRG_ERR_ARG, "null argument");
    for (int k = 0; k < 3; ++k) {
      order3[k] = b->order[k];
      if (ms9)
        for (int o = 0; o < 3; ++o) ms9[3 * k + o] = b->ms[k][2 * o + (b->width[k] == 64 ? 1 : 0)];
    }
    return DMRG_OK;
  });
}

dmrg_status dmrg_batch_tuning(dmrg_batch* b, int32_t* order3, int32_t* width3, float* ms18) {
  return guard([&]() -> dmrg_status {
    if (!b || !order3 || !width3) return fail(DMRG_ERR_ARG, "null argument");
    for (int k = 0; k < 3; ++k) {
      order3[k] = b->order[k];
      width3[k] = b->width[k];
      if (ms18)
        for (int c = 0; c < 6; ++c) ms18[6 * k + c] = b->ms[k][c];
    }
    return DMRG_OK;
  });
}

void dmrg_batch_destroy(dmrg_batch* b) {
  if (!b) return;
  try {
    DmrgDeviceGuard dg(b->dead ? -1 : b->device);   // the merged plans live on the handles' device
    retire(b);
  } catch (...) {
  }
  delete b;
}

}  // extern "C"

void dmrg_internal_handle_gone(dmrg_handle* h) {
  // retire() edits h->batches: work on a copy
  const std::vector<dmrg_batch*> live = h->batches;
  for (dmrg_batch* b : live) {
    try {
      retire(b);
    } catch (...) {
      b->dead = true;
    }
  }
  h->batches.clear();
}
