// C ABI (include/dmrg_gb300.h) over the host core.  Every entry point catches
// all exceptions and returns a status; messages are kept per thread.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>

#include <cuda_runtime.h>

#include "capi_internal.h"

namespace {
thread_local std::string g_err;

dmrg_status fail(dmrg_status s, const std::string& m) { return dmrg_internal_fail(s, m); }

template <class F>
dmrg_status guard(F&& f) {
  return dmrg_internal_guard(std::forward<F>(f));
}

// entry points on a handle run with the handle's device current (the device that
// was current at dmrg_build_ops); the caller's current device is restored on return
template <class F>
dmrg_status guard_h(dmrg_handle* h, F&& f) {
  return dmrg_internal_guard_on(h ? h->device : -1, std::forward<F>(f));
}

bool finite(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

dmrg_status check_device(dmrg_handle* h) { return dmrg_internal_check_device(h); }

// the handle's integrals in the caller's numbering from the engine's chain-order ones
// (after orbital rotations of the mode optimisation)
void sync_user_integrals(dmrg_handle* h) {
  const int L = h->L;
  const std::vector<int>& o = h->eng->problem().ord;
  const std::vector<double>& tc = h->eng->chain_t();
  const std::vector<double>& vc = h->eng->chain_v();
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) h->t_user[size_t(o[i]) * L + o[j]] = tc[size_t(i) * L + j];
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j)
      for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l)
          h->v_user[((size_t(o[i]) * L + o[j]) * L + o[k]) * L + o[l]] = vc[((size_t(i) * L + j) * L + k) * L + l];
}

// integrals in the caller's numbering -> chain order (position i holds orbital ord[i])
void to_chain(int L, const std::vector<int>& ord, const double* t, const double* v, std::vector<double>& tc,
              std::vector<double>& vc) {
  const size_t L2 = size_t(L) * L;
  tc.resize(L2);
  vc.resize(L2 * L2);
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) tc[size_t(i) * L + j] = t[size_t(ord[i]) * L + ord[j]];
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j)
      for (int k = 0; k < L; ++k)
        for (int l = 0; l < L; ++l)
          vc[((size_t(i) * L + j) * L + k) * L + l] = v[((size_t(ord[i]) * L + ord[j]) * L + ord[k]) * L + ord[l]];
}

dmrg_status ensure_bond(dmrg_handle* h, int bond) {
  if (bond < 0 || bond > h->L - 2) return fail(DMRG_ERR_ARG, "bond out of range");
  if (h->eng->bond() != bond) {
    h->eng->build_left_blocks(bond);
    h->eng->build_right_blocks(bond + 2);
    h->eng->prepare_bond(bond);
  }
  return DMRG_OK;
}
}  // namespace

extern "C" {

dmrg_status dmrg_build_ops(const dmrg_problem* p, void* stream, dmrg_handle** out) {
  return guard([&]() -> dmrg_status {
    if (!p || !out) return fail(DMRG_ERR_ARG, "null argument");
    *out = nullptr;
    const int L = p->L;
    if (L < 2 || L > 64) return fail(DMRG_ERR_ARG, "L must be in [2, 64]");
    if (p->n_alpha < 0 || p->n_beta < 0 || p->n_alpha > L || p->n_beta > L)
      return fail(DMRG_ERR_ARG, "electron counts out of range");
    if (!p->t || !p->v) return fail(DMRG_ERR_ARG, "t and v are required");
    if (p->precision != DMRG_PREC_FP64 && p->precision != DMRG_PREC_MIXED_BF16)
      return fail(DMRG_ERR_ARG, "unknown precision");
    const size_t L2 = size_t(L) * L, L4 = L2 * L2;
    if (!finite(p->t, L2) || !finite(p->v, L4)) return fail(DMRG_ERR_NONFINITE, "non-finite integrals");
    std::vector<int> ord(L);
    for (int i = 0; i < L; ++i) ord[i] = p->order ? p->order[i] : i;
    {
      std::vector<int> seen(L, 0);
      for (int i = 0; i < L; ++i) {
        if (ord[i] < 0 || ord[i] >= L || seen[ord[i]]) return fail(DMRG_ERR_ARG, "order is not a permutation");
        seen[ord[i]] = 1;
      }
    }
    dmrg::Problem P;
    P.L = L;
    P.na = p->n_alpha;
    P.nb = p->n_beta;
    P.D = p->D > 0 ? p->D : 256;
    P.seed = p->seed;
    P.precision = p->precision;
    P.mem_cap = p->mem_cap_bytes;
    P.ord = ord;
    to_chain(L, ord, p->t, p->v, P.t, P.v);
    auto h = std::make_unique<dmrg_handle>();
    h->L = L;
    h->t_user.assign(p->t, p->t + L2);
    h->v_user.assign(p->v, p->v + L4);
    cudaGetDevice(&h->device);
    h->right_loaded = L;
    h->ex.reset(dmrg::make_cuda_exec(stream, p->precision));
    h->eng = std::make_unique<dmrg::Engine>(P, h->ex.get());
    *out = h.release();
    return DMRG_OK;
  });
}

dmrg_status dmrg_load_site(dmrg_handle* h, int32_t site, int32_t side, int32_t n_sectors,
                           const int32_t* sectors, const double* data) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !sectors || !data || n_sectors <= 0) return fail(DMRG_ERR_ARG, "null argument");
    if (site < 0 || site >= h->L) return fail(DMRG_ERR_ARG, "site out of range");
    dmrg::Sectors s;
    for (int k = 0; k < n_sectors; ++k) {
      s.q.push_back(dmrg::QN{sectors[3 * k], sectors[3 * k + 1]});
      s.dim.push_back(sectors[3 * k + 2]);
      if (sectors[3 * k + 2] <= 0) return fail(DMRG_ERR_ARG, "sector dimension must be positive");
      if (k > 0 && !(s.q[k - 1] < s.q[k])) return fail(DMRG_ERR_ARG, "sectors must be strictly ascending");
    }
    if (side == 0) {
      if (site != h->left_loaded) return fail(DMRG_ERR_ARG, "left sites must be loaded in order 0, 1, ...");
    } else if (side == 1) {
      if (site != h->right_loaded - 1) return fail(DMRG_ERR_ARG, "right sites must be loaded in order L-1, L-2, ...");
    } else {
      return fail(DMRG_ERR_ARG, "side must be 0 or 1");
    }
    // rows of each isometry come from the enlarged block; the engine validates them
    dmrg::Enlarged E;
    const dmrg::Block& prev = side == 0 ? h->eng->left_block(site) : h->eng->right_block(site + 1);
    E.build(prev.sec, side == 0);
    std::vector<const double*> mats;
    size_t off = 0;
    for (int k = 0; k < n_sectors; ++k) {
      int c = E.coarse.find(s.q[k]);
      if (c < 0) return fail(DMRG_ERR_ARG, "sector not reachable from the neighbouring block");
      if (s.dim[k] > E.coarse.dim[c]) return fail(DMRG_ERR_ARG, "isometry wider than the enlarged sector");
      mats.push_back(data + off);
      size_t n = size_t(E.coarse.dim[c]) * s.dim[k];
      if (!finite(data + off, n)) return fail(DMRG_ERR_NONFINITE, "non-finite isometry");
      off += n;
    }
    if (side == 0) {
      h->eng->load_left(site, s, mats);
      h->left_loaded = site + 1;
    } else {
      h->eng->load_right(site, s, mats);
      h->right_loaded = site;
    }
    h->any_loaded = true;
    return DMRG_OK;
  });
}

dmrg_status dmrg_prepare(dmrg_handle* h, int32_t bond) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h) return fail(DMRG_ERR_ARG, "null handle");
    if (bond < 0 || bond > h->L - 2) return fail(DMRG_ERR_ARG, "bond out of range");
    if (!h->eng->left_buildable(bond)) return fail(DMRG_ERR_ARG, "left sites 0..bond-1 are not loaded");
    if (!h->eng->right_buildable(bond + 2)) return fail(DMRG_ERR_ARG, "right sites bond+2..L-1 are not loaded");
    h->eng->build_left_blocks(bond);
    h->eng->build_right_blocks(bond + 2);
    h->eng->prepare_bond(bond);
    h->eng->exec()->sync();
    return DMRG_OK;
  });
}

dmrg_status dmrg_layout(dmrg_handle* h, int32_t bond, int32_t* n_blocks, const int64_t** table,
                        int64_t* psi_size) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !n_blocks || !table) return fail(DMRG_ERR_ARG, "null argument");
    if (h->eng->bond() != bond) return fail(DMRG_ERR_ARG, "bond not prepared (call dmrg_prepare)");
    *n_blocks = int32_t(h->eng->layout().size() / 7);
    *table = h->eng->layout().data();
    if (psi_size) *psi_size = h->eng->psi_size();
    return DMRG_OK;
  });
}

dmrg_status dmrg_sigma(dmrg_handle* h, int32_t bond, const double* psi, double* sig) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi || !sig) return fail(DMRG_ERR_ARG, "null argument");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    h->eng->sigma_precision(psi, sig, h->eng->problem().precision);
    h->eng->exec()->sync();
    return check_device(h);
  });
}

dmrg_status dmrg_sigma_ex(dmrg_handle* h, int32_t bond, const double* psi, double* sig, int32_t precision) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi || !sig) return fail(DMRG_ERR_ARG, "null argument");
    if (precision != DMRG_PREC_FP64 && precision != DMRG_PREC_MIXED_BF16) return fail(DMRG_ERR_ARG, "unknown precision");
    if (precision == DMRG_PREC_MIXED_BF16 && h->eng->problem().precision != DMRG_PREC_MIXED_BF16)
      return fail(DMRG_ERR_ARG, "the handle was not created with the split-BF16 precision");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    h->eng->sigma_precision(psi, sig, precision);
    h->eng->exec()->sync();
    return check_device(h);
  });
}

dmrg_status dmrg_sigma_host(dmrg_handle* h, int32_t bond, const double* psi, double* sig) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi || !sig) return fail(DMRG_ERR_ARG, "null argument");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    dmrg::Exec* ex = h->eng->exec();
    const size_t bytes = size_t(h->eng->psi_size()) * sizeof(double);
    double* d = static_cast<double*>(ex->alloc(2 * bytes));
    ex->h2d(d, psi, bytes);
    h->eng->sigma_precision(d, d + h->eng->psi_size(), h->eng->problem().precision);
    ex->d2h(sig, d + h->eng->psi_size(), bytes);
    ex->sync();
    ex->release(d);
    return check_device(h);
  });
}

dmrg_status dmrg_davidson(dmrg_handle* h, int32_t bond, double* psi, double tol, int32_t max_iter,
                          double* energy, int32_t* iterations) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi) return fail(DMRG_ERR_ARG, "null argument");
    if (!(tol > 0)) return fail(DMRG_ERR_ARG, "tol must be positive");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    int it = 0;
    double e = h->eng->davidson(psi, tol, max_iter > 0 ? max_iter : 100, 24, &it, 1);
    h->eng->exec()->sync();
    if (energy) *energy = e;
    if (iterations) *iterations = it;
    if (check_device(h) != DMRG_OK) return DMRG_ERR_TIMEOUT;
    if (!std::isfinite(e)) return fail(DMRG_ERR_NONFINITE, "non-finite energy");
    if (h->eng->last_rnorm > tol) return fail(DMRG_ERR_NOCONV, "Davidson did not reach the tolerance");
    return DMRG_OK;
  });
}

dmrg_status dmrg_sweep_ex(dmrg_handle* h, int32_t n_sweeps, const int32_t* D_schedule, double tol,
                          double* energies, int32_t flags, int32_t max_iter) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || n_sweeps <= 0) return fail(DMRG_ERR_ARG, "bad arguments");
    if (h->L < 3) return fail(DMRG_ERR_ARG, "sweeps need L >= 3");
    if (!(tol > 0)) return fail(DMRG_ERR_ARG, "tol must be positive");
    if (flags & ~7) return fail(DMRG_ERR_ARG, "unknown sweep flags");
    std::vector<int> D(n_sweeps);
    for (int s = 0; s < n_sweeps; ++s) {
      D[s] = D_schedule ? D_schedule[s] : h->eng->problem().D;
      if (D[s] <= 0) return fail(DMRG_ERR_ARG, "D must be positive");
    }
    if (h->any_loaded && !h->eng->right_buildable(2))
      return fail(DMRG_ERR_ARG, "a partially loaded basis must reach site 2 for sweeps");
    h->eng->set_D(D[0]);
    std::vector<double> e = h->eng->run_sweeps(n_sweeps, D.data(), tol, flags, max_iter > 0 ? max_iter : 100);
    h->eng->exec()->sync();
    if (flags & 6) sync_user_integrals(h);
    if (energies)
      for (int s = 0; s < n_sweeps; ++s) energies[s] = e[s];
    dmrg_status ds = check_device(h);
    if (ds != DMRG_OK) return ds;
    for (double x : e)
      if (!std::isfinite(x)) return fail(DMRG_ERR_NONFINITE, "non-finite energy");
    int nc = 0;
    for (const auto& lg : h->eng->sweep_log_)
      if (lg.status == 2) ++nc;
    if (nc)
      return fail(DMRG_ERR_NOCONV, std::to_string(nc) + " sweep step(s) reached max_iter without convergence "
                                   "(energies are written; dmrg_sweep_log lists the steps)");
    return DMRG_OK;
  });
}

dmrg_status dmrg_sweep(dmrg_handle* h, int32_t n_sweeps, const int32_t* D_schedule, double tol,
                       double* energies) {
  return dmrg_sweep_ex(h, n_sweeps, D_schedule, tol, energies, 0, 100);
}

dmrg_status dmrg_sweep_log(dmrg_handle* h, int32_t* n_steps, const double** rows, int32_t* n_kept,
                           const int32_t** kept) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !n_steps || !rows || !n_kept || !kept) return fail(DMRG_ERR_ARG, "null argument");
    const auto& lg = h->eng->sweep_log_;
    h->log_rows.clear();
    h->log_kept.clear();
    for (size_t k = 0; k < lg.size(); ++k) {
      const auto& x = lg[k];
      for (double v : {double(x.sweep), double(x.bond), double(x.ltr), double(x.iters), double(x.status), x.energy,
                       x.rnorm, x.discarded})
        h->log_rows.push_back(v);
      for (size_t j = 0; j + 2 < x.kept.size(); j += 3)
        for (int v : {int(k), x.kept[j], x.kept[j + 1], x.kept[j + 2]}) h->log_kept.push_back(v);
    }
    *n_steps = int32_t(lg.size());
    *rows = h->log_rows.data();
    *n_kept = int32_t(h->log_kept.size() / 4);
    *kept = h->log_kept.data();
    return DMRG_OK;
  });
}

dmrg_status dmrg_sweep_phases(dmrg_handle* h, double* seconds5) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !seconds5) return fail(DMRG_ERR_ARG, "bad arguments");
    for (int k = 0; k < 5; ++k) seconds5[k] = h->eng->phase_s[k];
    return DMRG_OK;
  });
}

dmrg_status dmrg_sigma_backward(dmrg_handle* h, int32_t bond, const double* psi, const double* lam,
                                double* g1, double* g2) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi || !lam || !g1 || !g2) return fail(DMRG_ERR_ARG, "null argument");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    const int L = h->L;
    const size_t L2 = size_t(L) * L, L4 = L2 * L2;
    std::vector<double> raw;
    h->eng->integral_gradient(lam, psi, raw);
    s = check_device(h);
    if (s != DMRG_OK) return s;
    // symmetric parts in the caller's numbering: g1 = sym2(dF/dt), g2 = 2 sym8(dF/dv)
    const std::vector<int>& o = h->eng->problem().ord;
    std::vector<double> a1(L2), a2(L4);
    dmrg::Exec* ex = h->eng->exec();
    ex->d2h(a1.data(), g1, L2 * sizeof(double));
    ex->d2h(a2.data(), g2, L4 * sizeof(double));
    auto T = [&](int i, int j) { return raw[size_t(i) * L + j]; };
    auto V = [&](int i, int j, int k, int l) { return raw[L2 + ((size_t(i) * L + j) * L + k) * L + l]; };
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j) a1[size_t(o[i]) * L + o[j]] += 0.5 * (T(i, j) + T(j, i));
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < L; ++j)
        for (int k = 0; k < L; ++k)
          for (int l = 0; l < L; ++l) {
            const double x = V(i, j, k, l) + V(j, i, k, l) + V(i, j, l, k) + V(j, i, l, k) + V(k, l, i, j) +
                             V(l, k, i, j) + V(k, l, j, i) + V(l, k, j, i);
            a2[((size_t(o[i]) * L + o[j]) * L + o[k]) * L + o[l]] += 0.25 * x;
          }
    for (double x : raw)
      if (!std::isfinite(x)) return fail(DMRG_ERR_NONFINITE, "non-finite derivative");
    ex->h2d(g1, a1.data(), L2 * sizeof(double));
    ex->h2d(g2, a2.data(), L4 * sizeof(double));
    ex->sync();
    return DMRG_OK;
  });
}

dmrg_status dmrg_set_integrals(dmrg_handle* h, const double* t, const double* v) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !t || !v) return fail(DMRG_ERR_ARG, "null argument");
    const int L = h->L;
    const size_t L2 = size_t(L) * L, L4 = L2 * L2;
    if (!finite(t, L2) || !finite(v, L4)) return fail(DMRG_ERR_NONFINITE, "non-finite integrals");
    std::vector<double> tc, vc;
    to_chain(L, h->eng->problem().ord, t, v, tc, vc);
    h->eng->set_integrals(tc, vc);
    h->t_user.assign(t, t + L2);
    h->v_user.assign(v, v + L4);
    return DMRG_OK;
  });
}

dmrg_status dmrg_sweep_state(dmrg_handle* h, int32_t* bond, int64_t* psi_size, double* psi_dev) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !bond || !psi_size) return fail(DMRG_ERR_ARG, "null argument");
    const double* p = h->eng->sweep_psi();
    if (!p || h->eng->bond() < 0) return fail(DMRG_ERR_ARG, "no swept state (call dmrg_sweep first)");
    *bond = h->eng->bond();
    *psi_size = h->eng->psi_size();
    if (psi_dev) {
      h->eng->exec()->d2d(psi_dev, p, size_t(h->eng->psi_size()) * sizeof(double));
      h->eng->exec()->sync();
    }
    return DMRG_OK;
  });
}

dmrg_status dmrg_set_state(dmrg_handle* h, int32_t bond, const double* psi) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi) return fail(DMRG_ERR_ARG, "null argument");
    if (h->eng->bond() != bond) return fail(DMRG_ERR_ARG, "bond not prepared (call dmrg_prepare)");
    h->eng->set_state(psi);
    return DMRG_OK;
  });
}

dmrg_status dmrg_expectation(dmrg_handle* h, int32_t bond, const double* lam, const double* psi, double* value) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !lam || !psi || !value) return fail(DMRG_ERR_ARG, "null argument");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    dmrg::Exec* ex = h->ex.get();
    const int64_t n = h->eng->psi_size();
    double* d = static_cast<double*>(ex->alloc(size_t(n + 1) * sizeof(double)));
    h->eng->sigma(psi, d);
    ex->mdot(lam, n, 1, d, n, 1, n, d + n, 1);
    ex->d2h(value, d + n, sizeof(double));
    ex->release(d);
    s = check_device(h);
    if (s != DMRG_OK) return s;
    if (!std::isfinite(*value)) return fail(DMRG_ERR_NONFINITE, "non-finite expectation value");
    return DMRG_OK;
  });
}

dmrg_status dmrg_orbital_gradient(dmrg_handle* h, const double* g1, const double* g2, double* grad) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !g1 || !g2 || !grad) return fail(DMRG_ERR_ARG, "null argument");
    dmrg::Exec* ex = h->ex.get();
    const int L = h->L;
    const size_t L2 = size_t(L) * L, L4 = L2 * L2;
    double* d = static_cast<double*>(ex->alloc((L2 + L4) * sizeof(double)));
    ex->h2d(d, h->t_user.data(), L2 * sizeof(double));
    ex->h2d(d + L2, h->v_user.data(), L4 * sizeof(double));
    ex->orbital_gradient(L, d, d + L2, g1, g2, grad);
    ex->sync();
    ex->release(d);
    return DMRG_OK;
  });
}

dmrg_status dmrg_eigh_batch(dmrg_handle* h, int32_t nmat, const int32_t* n, double* A, double* w, double* Z) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !n || !A || !w || !Z) return fail(DMRG_ERR_ARG, "null argument");
    if (nmat <= 0) return fail(DMRG_ERR_ARG, "nmat must be positive");
    if (A == Z) return fail(DMRG_ERR_ARG, "A and Z must be different buffers");
    std::vector<double*> Av, wv, Zv;
    std::vector<int> nv;
    int64_t ao = 0, wo = 0;
    for (int32_t b = 0; b < nmat; ++b) {
      if (n[b] <= 0 || n[b] > 6000) return fail(DMRG_ERR_ARG, "matrix order out of range (1..6000)");
      Av.push_back(A + ao);
      Zv.push_back(Z + ao);
      wv.push_back(w + wo);
      nv.push_back(n[b]);
      ao += int64_t(n[b]) * n[b];
      wo += n[b];
    }
    h->eng->exec()->syev(Av, wv, Zv, nv);
    h->eng->exec()->sync();
    return check_device(h);
  });
}

dmrg_status dmrg_two_site_rotate(dmrg_handle* h, int32_t bond, double theta, const double* psi, double* out) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi || !out) return fail(DMRG_ERR_ARG, "null argument");
    if (psi == out) return fail(DMRG_ERR_ARG, "psi and out must be different buffers");
    if (!std::isfinite(theta)) return fail(DMRG_ERR_ARG, "theta must be finite");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    h->eng->rotate_two_site(theta, psi, out);
    h->eng->exec()->sync();
    return DMRG_OK;
  });
}

dmrg_status dmrg_half_renyi(dmrg_handle* h, int32_t bond, const double* psi, double* s_half) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi || !s_half) return fail(DMRG_ERR_ARG, "null argument");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    *s_half = h->eng->half_renyi(psi);
    return check_device(h);
  });
}

dmrg_status dmrg_mode_step(dmrg_handle* h, double* theta, double* s_before, double* s_after) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !theta) return fail(DMRG_ERR_ARG, "null argument");
    if (!h->eng->sweep_psi() || h->eng->bond() < 0) return fail(DMRG_ERR_ARG, "no swept state (call dmrg_sweep first)");
    *theta = h->eng->mode_step(s_before, s_after);
    sync_user_integrals(h);
    return check_device(h);
  });
}

dmrg_status dmrg_get_integrals(dmrg_handle* h, double* t, double* v) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !t || !v) return fail(DMRG_ERR_ARG, "null argument");
    std::copy(h->t_user.begin(), h->t_user.end(), t);
    std::copy(h->v_user.begin(), h->v_user.end(), v);
    return DMRG_OK;
  });
}

dmrg_status dmrg_mode_log(dmrg_handle* h, int32_t* n, const double** rows) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !n || !rows) return fail(DMRG_ERR_ARG, "null argument");
    h->log_rows.clear();
    for (const auto& m : h->eng->mode_log_)
      for (double x : {double(m.sweep), double(m.bond), m.theta, m.s_before, m.s_after}) h->log_rows.push_back(x);
    *n = int32_t(h->eng->mode_log_.size());
    *rows = h->log_rows.data();
    return DMRG_OK;
  });
}

dmrg_status dmrg_term_work(dmrg_handle* h, int32_t bond, int32_t* n_terms, int64_t* work) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !n_terms) return fail(DMRG_ERR_ARG, "null argument");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    const std::vector<int64_t> w = h->eng->term_work();
    *n_terms = int32_t(w.size());
    if (work) std::copy(w.begin(), w.end(), work);
    return DMRG_OK;
  });
}

dmrg_status dmrg_term_partition(int32_t n, const int64_t* work, int32_t world, int32_t* owner) {
  return guard([&]() -> dmrg_status {
    if (n < 0 || world <= 0 || (n > 0 && (!work || !owner))) return fail(DMRG_ERR_ARG, "bad arguments");
    for (int32_t i = 0; i < n; ++i)
      if (work[i] < 0) return fail(DMRG_ERR_ARG, "negative work");
    // longest processing time first: terms by decreasing work (ties: lower index
    // first), each to the least loaded rank (ties: lower rank)
    std::vector<int32_t> ord(n);
    for (int32_t i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
    std::vector<int64_t> load(world, 0);
    for (int32_t i : ord) {
      int32_t r = 0;
      for (int32_t k = 1; k < world; ++k)
        if (load[k] < load[r]) r = k;
      owner[i] = r;
      load[r] += work[i];
    }
    return DMRG_OK;
  });
}

dmrg_status dmrg_sigma_subset(dmrg_handle* h, int32_t bond, const double* psi, double* sig, const int32_t* owner,
                              int32_t rank) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !psi || !sig || !owner) return fail(DMRG_ERR_ARG, "null argument");
    dmrg_status s = ensure_bond(h, bond);
    if (s != DMRG_OK) return s;
    const size_t nt = h->eng->term_work().size();
    std::vector<char> own(nt, 0);
    for (size_t i = 0; i < nt; ++i) own[i] = owner[i] == rank ? 1 : 0;
    h->eng->sigma_subset(psi, sig, own);
    h->eng->exec()->sync();
    return check_device(h);
  });
}

dmrg_status dmrg_stats(dmrg_handle* h, int64_t* o) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !o) return fail(DMRG_ERR_ARG, "null argument");
    const dmrg::BondStats& s = h->eng->stats();
    o[0] = s.psi_size;
    o[1] = s.n_terms;
    o[2] = s.flops_stage1;
    o[3] = s.flops_stage2;
    o[4] = s.op_bytes;
    o[5] = s.n_gemm_problems;
    o[6] = s.n_gemm_segments;
    o[7] = s.launches_per_sigma;
    o[8] = s.mix_tiles1;
    o[9] = s.mix_steps1;
    o[10] = s.mix_tiles2;
    o[11] = s.mix_steps2;
    o[12] = s.mix_x_elems;
    o[13] = s.mix_plane_bytes;
    o[14] = h->eng->exec()->alloc_count();
    o[15] = s.n_chunks;
    return DMRG_OK;
  });
}

dmrg_status dmrg_plan_paths(dmrg_handle* h, int64_t* o) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !o) return fail(DMRG_ERR_ARG, "null argument");
    if (h->eng->bond() < 0) return fail(DMRG_ERR_ARG, "no bond prepared");
    const dmrg::BondStats& s = h->eng->stats();
    o[0] = s.n_chunks;
    o[1] = s.mix_chunks;
    o[2] = s.mix_parts;
    o[3] = s.mix_mode2;
    o[4] = s.mix_mode3;
    o[5] = s.max_rows;
    o[6] = s.mix_multirow;
    o[7] = s.n_terms;
    return DMRG_OK;
  });
}

dmrg_status dmrg_graph_replays(dmrg_handle* h, int64_t* replays) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h || !replays) return fail(DMRG_ERR_ARG, "null argument");
    *replays = h->eng->graph_runs();
    return DMRG_OK;
  });
}

dmrg_status dmrg_profile(dmrg_handle* h, int32_t mode, double* out) {
  return guard_h(h, [&]() -> dmrg_status {
    if (!h) return fail(DMRG_ERR_ARG, "null handle");
    if (mode != 0 && mode != 1) return fail(DMRG_ERR_ARG, "mode must be 0 or 1");
    h->eng->exec()->profile(mode, out);
    return DMRG_OK;
  });
}

void dmrg_destroy(dmrg_handle* h) {
  try {
    if (h) {
      DmrgDeviceGuard dg(h->device);   // the handle's memory lives on its device
      dmrg_internal_handle_gone(h);
      h->eng.reset();
      h->ex.reset();
      delete h;
    }
  } catch (...) {
  }
}

const char* dmrg_last_error(void) { return g_err.c_str(); }

}  // extern "C"

void dmrg_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }

extern "C" {

}  // extern "C"
