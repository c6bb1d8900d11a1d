// Engine: block construction from an MPS basis, Davidson (Fig. 1 i: iterative
// eigensolver for the effective Hamiltonian), density-matrix truncation
// (keep the D largest weights, Sec. 2.1), renormalisation Ren_l / Ren_r and the
// wave-function transformation StVec of the two-site sweep (Sec. 4.1).
#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "core.h"

namespace dmrg {

Engine::Engine(const Problem& p, Exec* ex) : P_(p), ex_(ex) {
  if (P_.L < 2) throw std::runtime_error("L must be >= 2");
  lb_.resize(P_.L + 1);
  rb_.resize(P_.L + 1);
  liso_.resize(P_.L);
  riso_.resize(P_.L);
  // vacuum blocks B_0 and C_L: one state (0,0), H = 0
  for (Block* b : {&lb_[0], &rb_[P_.L]}) {
    b->sec.q = {QN{0, 0}};
    b->sec.dim = {1};
    b->sec.finalize();
    b->valid = true;
  }
  auto vac_ops = [&](Block& b, bool left) {
    std::vector<OpKey> keys = left ? std::vector<OpKey>() : std::vector<OpKey>();
    OpKey hk{OP_H, 0, 0};
    Op h;
    h.blk.push_back(OpBlk{0, 0, 1, 1, 0, 0});
    h.by_col[0] = 0;
    h.by_row[0] = 0;
    b.ops.ops[hk] = h;
    (void)left;  // every other operator of the vacuum is zero (absent)
    alloc_opset(b.ops);
    ex_->zero(b.ops.arena, b.ops.n_elem * sizeof(double));
  };
  vac_ops(lb_[0], true);
  vac_ops(rb_[P_.L], false);
}

Engine::~Engine() {
  free_bond();
  for (auto& b : lb_) free_opset(b.ops);
  for (auto& b : rb_) free_opset(b.ops);
  for (auto* v : {&liso_, &riso_})
    for (auto& i : *v)
      if (i.arena) ex_->release(i.arena);
  if (psi_cur_) ex_->release(psi_cur_);
}

static void set_iso(Exec* ex, Iso& iso, const Sectors& out, const std::vector<int>& rows,
                    const std::vector<const double*>& mats, bool device_src) {
  if (iso.arena) ex->release(iso.arena);
  iso.out = out;
  iso.out.finalize();
  iso.rows = rows;
  int64_t n = 0;
  for (size_t k = 0; k < out.q.size(); ++k) n += int64_t(rows[k]) * out.dim[k];
  iso.arena = static_cast<double*>(ex->alloc(std::max<int64_t>(n, 1) * sizeof(double)));
  iso.mat.assign(out.q.size(), nullptr);
  int64_t o = 0;
  for (size_t k = 0; k < out.q.size(); ++k) {
    iso.mat[k] = iso.arena + o;
    size_t bytes = size_t(rows[k]) * out.dim[k] * sizeof(double);
    if (mats[k]) {
      if (device_src) ex->d2d(iso.mat[k], mats[k], bytes);
      else ex->h2d(iso.mat[k], mats[k], bytes);
    }
    o += int64_t(rows[k]) * out.dim[k];
  }
  iso.valid = true;
}

static std::vector<int> iso_rows(const Sectors& prev, const Sectors& out) {
  Enlarged E;
  E.build(prev, true);
  std::vector<int> rows(out.q.size());
  for (size_t k = 0; k < out.q.size(); ++k) {
    int c = E.coarse.find(out.q[k]);
    if (c < 0) throw std::runtime_error("isometry: sector not reachable from the previous block");
    rows[k] = E.coarse.dim[c];
  }
  return rows;
}

void Engine::load_left(int site, const Sectors& out, const std::vector<const double*>& mats) {
  if (site < 0 || site >= P_.L) throw std::runtime_error("load_left: site out of range");
  if (lb_[site].sec.q.empty()) throw std::runtime_error("load_left: previous left block sectors unknown");
  Sectors o = out;
  o.finalize();
  set_iso(ex_, liso_[site], o, iso_rows(lb_[site].sec, o), mats, false);
  // record the sector table of B_{site+1} so that the next site can be loaded
  free_opset(lb_[site + 1].ops);
  lb_[site + 1].sec = o;
  lb_[site + 1].valid = false;
  // mark sectors known (ops not yet built)
  lb_[site + 1].ops.ops.clear();
  lb_sec_known_ = std::max(lb_sec_known_, site + 1);
}

void Engine::load_right(int site, const Sectors& out, const std::vector<const double*>& mats) {
  if (site < 0 || site >= P_.L) throw std::runtime_error("load_right: site out of range");
  Sectors o = out;
  o.finalize();
  const Sectors& prev = rb_[site + 1].sec;
  if (prev.q.empty()) throw std::runtime_error("load_right: next right block sectors unknown");
  set_iso(ex_, riso_[site], o, iso_rows(prev, o), mats, false);
  free_opset(rb_[site].ops);
  rb_[site].sec = o;
  rb_[site].valid = false;
}

bool Engine::left_buildable(int n) const {
  for (int k = n; k >= 0; --k) {
    if (lb_[k].valid) return true;
    if (k == 0 || !liso_[k - 1].valid) return false;
  }
  return false;
}

bool Engine::right_buildable(int m) const {
  for (int k = m; k <= P_.L; ++k) {
    if (rb_[k].valid) return true;
    if (k == P_.L || !riso_[k].valid) return false;
  }
  return false;
}

void Engine::build_left_blocks(int upto) {
  for (int n = 0; n < upto; ++n) {
    if (lb_[n + 1].valid) continue;
    if (!liso_[n].valid) throw std::runtime_error("build_left_blocks: missing isometry");
    Enlarged E;
    OpSet eops;
    enlarge(true, lb_[n], n, E, eops);
    renormalize(true, E, eops, liso_[n], lb_[n + 1]);
    free_opset(eops);
  }
}

void Engine::build_right_blocks(int downto) {
  for (int m = P_.L - 1; m >= downto; --m) {
    if (rb_[m].valid) continue;
    if (!riso_[m].valid) throw std::runtime_error("build_right_blocks: missing isometry");
    Enlarged E;
    OpSet eops;
    enlarge(false, rb_[m + 1], m, E, eops);
    renormalize(false, E, eops, riso_[m], rb_[m]);
    free_opset(eops);
  }
}

// ---------------------------------------------------------------------------
// Davidson (FP64 subspace, Gram-Schmidt twice, Rayleigh-Ritz on the device)

double Engine::davidson(double* psi, double tol, int max_iter, int max_sub, int* iters_out, int refine) {
  if (bond_ < 0) throw std::runtime_error("davidson: no bond prepared");
  const int64_t n = psi_n_;
  max_sub = std::max(3, std::min(max_sub, 32));
  double* V = static_cast<double*>(ex_->alloc(size_t(max_sub) * n * sizeof(double)));
  double* W = static_cast<double*>(ex_->alloc(size_t(max_sub) * n * sizeof(double)));
  double* x = static_cast<double*>(ex_->alloc(n * sizeof(double)));
  double* wx = static_cast<double*>(ex_->alloc(n * sizeof(double)));
  double* xp = static_cast<double*>(ex_->alloc(n * sizeof(double)));   // previous Ritz vector
  double* wxp = static_cast<double*>(ex_->alloc(n * sizeof(double)));
  bool have_prev = false;
  double* r = static_cast<double*>(ex_->alloc(n * sizeof(double)));
  double* t = static_cast<double*>(ex_->alloc(n * sizeof(double)));
  double* diag = static_cast<double*>(ex_->alloc(n * sizeof(double)));
  const int lds = 40;
  double* small = static_cast<double*>(ex_->alloc(size_t(lds) * lds * 2 * sizeof(double)));
  double* Hs = small;
  double* sc = small + lds * lds;  // scratch: [0] theta, [1] nrm2, [2..] coefficients / y
  double* theta = sc;
  double* nrm2 = sc + 1;
  double* y = sc + 8;
  double* cf = sc + 8 + lds;
  ex_->zero(small, size_t(lds) * lds * 2 * sizeof(double));
  diagonal(diag);
  const int prec = P_.precision;

  auto apply = [&](const double* in, double* out, int pr) {
    if (pr == 0) sigma(in, out);
    else sigma_precision(in, out, pr);
  };

  // v0 = normalised guess
  ex_->mdot(psi, n, 1, psi, n, 1, n, nrm2, 1);
  ex_->d2d(V, psi, n * sizeof(double));
  ex_->normalize(V, n, nrm2);
  apply(V, W, prec);
  int m = 1;
  ex_->mdot(V, n, 1, W, n, 1, n, Hs, lds);
  double rnorm = 1e300, th = 0.0;
  int it = 0;
  // Mixed precision: iterate with the split-BF16 sigma; when its residual reaches
  // the level that precision can resolve (or stalls), restart from the Ritz vector
  // x with an FP64 sigma W0 = H x (a refinement).  Right after a refinement the
  // residual W0 - theta x is exact, and only an exact residual can declare
  // convergence.  Later corrections V_i get split-BF16 sigmas, but their couplings
  // to x are taken from the exact pair (<V_i|H x> = <W0|V_i>, H symmetric), so the
  // corrections carry only the small error of their own small coefficients.
  const bool mixed = (prec != 0 && refine);
  int refines = 0, last_refine = -100;
  bool exact0 = false;   // W[0] is an FP64 sigma of V[0], up to the error w0err
  double w0err = 0.0;
  double best = 1e300;
  int best_it = 0;
  int status = 2;
  // second direction of a restart: the part of the previous Ritz vector orthogonal to
  // V[0] = x, kept only when well resolved (|xp - c x| > 1e-4) and orthogonalised once
  // more against x; with an exact W[0] its coupling comes from the exact pair
  auto second = [&](bool exact) {
    if (!have_prev) return;
    double* V1 = V + n;
    double* W1 = W + n;
    ex_->mdot(x, n, 1, xp, n, 1, n, cf, 1);
    ex_->d2d(V1, xp, n * sizeof(double));
    ex_->axpy_dev(x, V1, n, cf, -1.0);
    ex_->d2d(W1, wxp, n * sizeof(double));
    ex_->axpy_dev(wx, W1, n, cf, -1.0);
    ex_->mdot(V1, n, 1, V1, n, 1, n, nrm2, 1);
    double pn2;
    ex_->d2h(&pn2, nrm2, sizeof(double));
    if (!(pn2 > 1e-8)) return;
    ex_->normalize(V1, n, nrm2);
    ex_->normalize(W1, n, nrm2);
    ex_->mdot(V, n, 1, V1, n, 1, n, cf, 1);
    ex_->axpy_dev(V, V1, n, cf, -1.0);
    ex_->axpy_dev(W, W1, n, cf, -1.0);
    ex_->mdot(V1, n, 1, V1, n, 1, n, nrm2, 1);
    ex_->normalize(V1, n, nrm2);
    ex_->normalize(W1, n, nrm2);
    ex_->mdot(V, n, 2, W1, n, 1, n, Hs + 1, lds);
    if (exact) ex_->mdot(W, n, 1, V1, n, 1, n, Hs + 1, lds);
    m = 2;
  };
  for (;; ++it) {
    ex_->ritz(Hs, lds, m, theta, y);
    if (it > 0) {
      std::swap(x, xp);
      std::swap(wx, wxp);
      have_prev = true;
    }
    ex_->lincomb(V, n, m, y, 1, 1, n, x, n, 1.0, 0.0);
    ex_->lincomb(W, n, m, y, 1, 1, n, wx, n, 1.0, 0.0);
    ex_->d2d(r, wx, n * sizeof(double));
    ex_->axpy_dev(x, r, n, theta, -1.0);
    ex_->mdot(r, n, 1, r, n, 1, n, nrm2, 1);
    double h2[9];   // theta, |r|^2, (unused), y[0]
    ex_->d2h(h2, sc, 9 * sizeof(double));
    th = h2[0];
    rnorm = std::sqrt(std::max(0.0, h2[1]));
    const double y0 = h2[8];
    if (rnorm < 0.9 * best) {
      best = rnorm;
      best_it = it;
    }
    if (!mixed) {
      if (rnorm <= tol) {
        status = 0;
        break;
      }
      // split-BF16 sigma without refinement: its residual cannot fall below the
      // level that precision resolves; stop there instead of running to max_iter
      if (prec != 0) {
        const double floor_m = 1e-6 * std::max(1.0, std::fabs(th));
        if (rnorm <= floor_m || it - best_it >= 8) {
          status = 1;
          break;
        }
      }
    } else {
      const bool just_refined = (it == last_refine + 1);
      // the split-BF16 error of a computed residual: about 1e-6 |theta| per unit weight of
      // split-BF16 sigmas in it (all of it before a refinement or after a restart; only
      // the weight |y_1..| of the corrections while x = V[0] carries its exact sigma)
      const double floor_m = 1e-6 * std::max(1.0, std::fabs(th));
      const double floor_c = exact0 ? w0err + floor_m * std::sqrt(std::max(0.0, 1.0 - y0 * y0)) : floor_m;
      bool want;
      if (refines == 0 || !exact0)
        want = rnorm <= std::max(tol, floor_m) || it - best_it >= 8;
      else
        want = rnorm <= std::max(tol, 2.0 * floor_c) || (!just_refined && it - best_it >= 40);
      if (want && refines < 24) {
        ++refines;
        last_refine = it;
        best = 1e300;
        best_it = it;
        // x (and its split-BF16 sigma wx) normalised; V[0] = x with the exact W[0] = H x
        ex_->mdot(x, n, 1, x, n, 1, n, nrm2, 1);
        ex_->normalize(x, n, nrm2);
        ex_->normalize(wx, n, nrm2);
        ex_->d2d(V, x, n * sizeof(double));
        apply(V, W, 0);
        ex_->zero(Hs, size_t(lds) * lds * sizeof(double));
        ex_->mdot(V, n, 1, W, n, 1, n, Hs, lds);
        // the exact residual of x decides convergence
        ex_->d2d(theta, Hs, sizeof(double));
        ex_->d2d(r, W, n * sizeof(double));
        ex_->axpy_dev(V, r, n, theta, -1.0);
        ex_->mdot(r, n, 1, r, n, 1, n, nrm2, 1);
        double e2[2];
        ex_->d2h(e2, sc, 2 * sizeof(double));
        th = e2[0];
        rnorm = std::sqrt(std::max(0.0, e2[1]));
        if (rnorm <= tol) {
          status = 0;
          break;
        }
        m = 1;
        exact0 = true;
        w0err = 0.0;
        second(true);
        have_prev = false;
        continue;
      }
    }
    if (it >= max_iter) break;
    if (m == max_sub) {
      // restart with the current Ritz vector and the part of the previous one
      // orthogonal to it (two-vector restart)
      ex_->d2d(V, x, n * sizeof(double));
      ex_->d2d(W, wx, n * sizeof(double));
      ex_->zero(Hs, size_t(lds) * lds * sizeof(double));
      ex_->d2d(Hs, theta, sizeof(double));
      m = 1;
      // after a refinement the restart pair (x, wx) keeps W[0] = H x up to the split-BF16
      // error of its correction components, which the floor carries on
      if (exact0 && prec != 0) w0err += 1e-6 * std::max(1.0, std::fabs(th)) * std::sqrt(std::max(0.0, 1.0 - y0 * y0));
      second(exact0 && prec != 0);
    }
    ex_->precond(r, diag, theta, n, t, 1e-8);
    for (int pass = 0; pass < 2; ++pass) {
      ex_->mdot(V, n, m, t, n, 1, n, cf, 1);
      ex_->lincomb(V, n, m, cf, 1, 1, n, t, n, -1.0, 1.0);
    }
    ex_->mdot(t, n, 1, t, n, 1, n, nrm2, 1);
    double tn2;
    ex_->d2h(&tn2, nrm2, sizeof(double));
    if (!(tn2 > 1e-28)) {  // no new direction
      status = 3;
      break;
    }
    ex_->normalize(t, n, nrm2);
    ex_->d2d(V + int64_t(m) * n, t, n * sizeof(double));
    apply(V + int64_t(m) * n, W + int64_t(m) * n, prec);
    ex_->mdot(V, n, m + 1, W + int64_t(m) * n, n, 1, n, Hs + m, lds);
    if (exact0 && prec != 0) ex_->mdot(W, n, 1, V + int64_t(m) * n, n, 1, n, Hs + m, lds);
    ++m;
  }
  // normalised Ritz vector out
  ex_->mdot(x, n, 1, x, n, 1, n, nrm2, 1);
  ex_->normalize(x, n, nrm2);
  ex_->d2d(psi, x, n * sizeof(double));
  for (double* p : {V, W, x, wx, xp, wxp, r, t, diag, small}) ex_->release(p);
  if (iters_out) *iters_out = it + 1;
  last_energy = th;
  last_rnorm = rnorm;
  last_status = status;
  return th;
}

// ---------------------------------------------------------------------------
// truncation and moving the two-site window

namespace {

struct Weight {
  double w;
  int sec, idx;
};

// Keep at most D states: largest weights first, ties by (sector, index); never cut
// inside a group of weights closer than 1e-10 * w_max.
std::vector<int> select_kept(const std::vector<std::vector<double>>& w, int D, double* discarded) {
  std::vector<Weight> all;
  for (size_t s = 0; s < w.size(); ++s)
    for (size_t i = 0; i < w[s].size(); ++i) all.push_back(Weight{std::max(0.0, w[s][i]), int(s), int(i)});
  std::stable_sort(all.begin(), all.end(), [](const Weight& a, const Weight& b) {
    if (a.w != b.w) return a.w > b.w;
    if (a.sec != b.sec) return a.sec < b.sec;
    return a.idx < b.idx;
  });
  int nk = std::min<int>(D, int(all.size()));
  if (nk < int(all.size()) && !all.empty() && all[0].w > 0) {
    int k = nk;
    while (k > 0 && all[k - 1].w - all[k].w <= 1e-10 * all[0].w) --k;
    if (k > 0) nk = k;
  }
  std::vector<int> kept(w.size(), 0);
  double disc = 0.0;
  for (size_t i = 0; i < all.size(); ++i) {
    if (int(i) < nk) kept[all[i].sec]++;
    else disc += all[i].w;
  }
  if (discarded) *discarded = disc;
  return kept;
}

}  // namespace

void Engine::truncate_and_move(bool ltr, int D, double* trunc_w, std::vector<int>* kept_out) {
  const int b = bond_;
  const Enlarged& E = ltr ? EL_ : ER_;
  const int nc = int(E.coarse.q.size());
  // density matrices rho_i = psi psi^T (left) or psi^T psi (right) per coarse sector
  std::vector<int> sec_of, dims;
  std::vector<int64_t> roff;
  int64_t tot = 0, totw = 0;
  std::vector<int> blk_of(nc, -1);  // coarse -> left coarse index of the psi block
  for (size_t i = 0; i < EL_.coarse.q.size(); ++i) {
    if (psi_off_[i] < 0) continue;
    int c = ltr ? int(i) : psi_rcoarse_[i];
    blk_of[c] = int(i);
  }
  for (int c = 0; c < nc; ++c) {
    if (blk_of[c] < 0) continue;
    sec_of.push_back(c);
    dims.push_back(E.coarse.dim[c]);
    roff.push_back(tot);
    tot += int64_t(E.coarse.dim[c]) * E.coarse.dim[c];
    totw += E.coarse.dim[c];
  }
  const int ns = int(sec_of.size());
  double* rho = static_cast<double*>(ex_->alloc(size_t(tot) * sizeof(double)));
  double* Z = static_cast<double*>(ex_->alloc(size_t(tot) * sizeof(double)));
  double* wv = static_cast<double*>(ex_->alloc(size_t(totw) * sizeof(double)));
  {
    std::vector<GemmProb> P;
    std::vector<GemmSeg> S;
    for (int k = 0; k < ns; ++k) {
      int i = blk_of[sec_of[k]];
      const double* A = psi_cur_ + psi_off_[i];
      int rows = EL_.coarse.dim[i], cols = ER_.coarse.dim[psi_rcoarse_[i]];
      GemmProb q;
      q.C = rho + roff[k];
      q.ldc = dims[k];
      q.M = dims[k];
      q.N = dims[k];
      q.alpha = 1.0;
      q.accumulate = 0;
      q.s0 = int(S.size());
      if (ltr) S.push_back(GemmSeg{A, A, cols, cols, cols, 0, 1});
      else S.push_back(GemmSeg{A, A, cols, cols, rows, 1, 0});
      q.s1 = int(S.size());
      P.push_back(q);
    }
    ex_->gemm(P, S);
  }
  {
    std::vector<double*> Av, wvv, Zv;
    std::vector<int> nv;
    int64_t wo = 0;
    for (int k = 0; k < ns; ++k) {
      Av.push_back(rho + roff[k]);
      Zv.push_back(Z + roff[k]);
      wvv.push_back(wv + wo);
      nv.push_back(dims[k]);
      wo += dims[k];
    }
    ex_->syev(Av, wvv, Zv, nv);
    tick(2);
  }
  std::vector<double> hw(totw);
  ex_->d2h(hw.data(), wv, totw * sizeof(double));
  std::vector<std::vector<double>> w(ns);
  {
    int64_t wo = 0;
    for (int k = 0; k < ns; ++k) {
      w[k].assign(hw.begin() + wo, hw.begin() + wo + dims[k]);
      wo += dims[k];
    }
  }
  double disc = 0.0;
  std::vector<int> kept = select_kept(w, D, &disc);
  if (trunc_w) *trunc_w = disc;
  // new block sectors and isometry (kept eigenvectors: last columns of ascending Z)
  Sectors out;
  std::vector<int> krow;   // rows of each kept sector's isometry
  std::vector<int> kk;     // index k into sec_of
  for (int k = 0; k < ns; ++k)
    if (kept[k] > 0) {
      out.q.push_back(E.coarse.q[sec_of[k]]);
      out.dim.push_back(kept[k]);
      krow.push_back(dims[k]);
      kk.push_back(k);
    }
  out.finalize();
  if (kept_out) {
    kept_out->clear();
    for (size_t k = 0; k < out.q.size(); ++k) {
      kept_out->push_back(out.q[k].a);
      kept_out->push_back(out.q[k].b);
      kept_out->push_back(out.dim[k]);
    }
  }
  Iso& iso = ltr ? liso_[b] : riso_[b + 1];
  std::vector<const double*> nulls(out.q.size(), nullptr);
  set_iso(ex_, iso, out, krow, nulls, true);
  {
    std::vector<KronGroup> g;
    std::vector<KronTask> t;
    for (size_t s = 0; s < out.q.size(); ++s) {
      int k = kk[s];
      KronGroup gg;
      gg.dst = iso.mat[s];
      gg.ld = out.dim[s];
      gg.rows = dims[k];
      gg.cols = out.dim[s];
      gg.t0 = int(t.size());
      gg.accumulate = 0;
      t.push_back(KronTask{Z + roff[k] + (dims[k] - kept[k]), dims[k], 0, 1.0});
      gg.t1 = int(t.size());
      g.push_back(gg);
    }
    ex_->kron(g, t);
  }
  ex_->release(rho);
  ex_->release(Z);
  ex_->release(wv);

  // Y = U^T psi (left) or psi V (right), block (kept sector, partner coarse)
  std::vector<int64_t> yoff(E.coarse.q.size(), -1);
  std::vector<int> ycols(E.coarse.q.size(), 0);
  int64_t ytot = 0;
  for (size_t s = 0; s < out.q.size(); ++s) {
    int c = sec_of[kk[s]];
    int i = blk_of[c];
    int partner_dim = ltr ? ER_.coarse.dim[psi_rcoarse_[i]] : EL_.coarse.dim[i];
    yoff[c] = ytot;
    ycols[c] = partner_dim;
    ytot += int64_t(out.dim[s]) * partner_dim;
  }
  double* Y = static_cast<double*>(ex_->alloc(std::max<int64_t>(ytot, 1) * sizeof(double)));
  {
    std::vector<GemmProb> P;
    std::vector<GemmSeg> S;
    for (size_t s = 0; s < out.q.size(); ++s) {
      int c = sec_of[kk[s]];
      int i = blk_of[c];
      const double* A = psi_cur_ + psi_off_[i];
      int rows = EL_.coarse.dim[i], cols = ER_.coarse.dim[psi_rcoarse_[i]];
      GemmProb q;
      q.alpha = 1.0;
      q.accumulate = 0;
      q.s0 = int(S.size());
      if (ltr) {  // Y (kept x cols) = U^T psi
        q.C = Y + yoff[c];
        q.ldc = cols;
        q.M = out.dim[s];
        q.N = cols;
        S.push_back(GemmSeg{iso.mat[s], A, out.dim[s], cols, rows, 1, 0});
      } else {    // Y stored transposed: (kept x rows) = V^T psi^T
        q.C = Y + yoff[c];
        q.ldc = rows;
        q.M = out.dim[s];
        q.N = rows;
        S.push_back(GemmSeg{iso.mat[s], A, out.dim[s], cols, cols, 1, 1});
      }
      q.s1 = int(S.size());
      P.push_back(q);
    }
    ex_->gemm(P, S);
  }
  // renormalise the operators of the enlarged block that was truncated
  Enlarged Eold = E;
  tick(2);
  if (ltr) {
    renormalize(true, EL_, EopsL_, iso, lb_[b + 1]);
  } else {
    renormalize(false, ER_, EopsR_, iso, rb_[b + 1]);
  }
  tick(3);
  Enlarged ELold = EL_, ERold = ER_;
  std::vector<int64_t> old_poff = psi_off_;
  std::vector<int> old_prc = psi_rcoarse_;
  free_bond();

  // StVec: psi at the neighbouring bond
  const int nb = ltr ? b + 1 : b - 1;
  Enlarged EL2, ER2;
  EL2.build(lb_[nb].sec, true);
  ER2.build(rb_[nb + 2].sec, false);
  QN N{P_.na, P_.nb};
  std::vector<int64_t> poff(EL2.coarse.q.size(), -1);
  std::vector<int> prc(EL2.coarse.q.size(), -1);
  int64_t pn = 0;
  for (size_t i = 0; i < EL2.coarse.q.size(); ++i) {
    int j = ER2.coarse.find(N - EL2.coarse.q[i]);
    if (j < 0) continue;
    poff[i] = pn;
    prc[i] = j;
    pn += int64_t(EL2.coarse.dim[i]) * ER2.coarse.dim[j];
  }
  double* npsi = static_cast<double*>(ex_->alloc(std::max<int64_t>(pn, 1) * sizeof(double)));
  ex_->zero(npsi, std::max<int64_t>(pn, 1) * sizeof(double));
  {
    std::vector<GemmProb> P;
    std::vector<GemmSeg> S;
    for (size_t i = 0; i < EL2.coarse.q.size(); ++i) {
      if (poff[i] < 0) continue;
      const int j = prc[i];
      const int cols = ER2.coarse.dim[j];
      for (int f : EL2.coarse_fines[i])
        for (int g : ER2.coarse_fines[j]) {
          const int s1 = EL2.f_s[f], s2 = ER2.f_s[g];
          GemmProb q;
          q.C = npsi + poff[i] + int64_t(EL2.f_row[f]) * cols + ER2.f_row[g];
          q.ldc = cols;
          q.M = EL2.f_dim[f];
          q.N = ER2.f_dim[g];
          q.alpha = 1.0;
          q.accumulate = 0;
          q.s0 = int(S.size());
          if (ltr) {
            // psi'[(k,s1),(s2,c')] = sum_c Y[k,(s1,c)] V_{b+2}[(s2,c'),c]
            const int k = EL2.f_part[f];                 // B_{b+1} sector (new block)
            const QN Qc = kLocalQ[s2] + rb_[nb + 2].sec.q[ER2.f_part[g]];
            const int cidx = rb_[b + 2].sec.find(Qc);
            if (cidx < 0) { q.s1 = q.s0; P.push_back(q); continue; }
            const int cY = Eold.coarse.find(lb_[nb].sec.q[k]);  // old L' coarse = kept sector
            const int jR = ERold.coarse.find(kLocalQ[s1] + Qc);
            const int fcol = ERold.part_s_to_fine[cidx][s1];
            if (cY < 0 || yoff[cY] < 0 || jR < 0 || old_prc[blk_of[cY]] != jR) { q.s1 = q.s0; P.push_back(q); continue; }
            const Iso& V = riso_[b + 2];
            const int vk = V.out.find(Qc);
            const int dimc = rb_[b + 2].sec.dim[cidx];
            S.push_back(GemmSeg{Y + yoff[cY] + ERold.f_row[fcol], V.mat[vk] + int64_t(ER2.f_row[g]) * dimc,
                                ycols[cY], dimc, dimc, 0, 1});
          } else {
            // psi'[(a',s1),(s2,k)] = sum_alpha U_{b-1}[(a',s1),alpha] Y^T[(alpha,s2),k]
            const int k = ER2.f_part[g];                 // C_{b+1} sector (new block)
            const QN Qa = lb_[nb].sec.q[EL2.f_part[f]] + kLocalQ[s1];
            const int aidx = lb_[b].sec.find(Qa);
            if (aidx < 0) { q.s1 = q.s0; P.push_back(q); continue; }
            const int cY = Eold.coarse.find(rb_[nb + 2].sec.q[k]);  // old R' coarse = kept sector
            const int iL = ELold.coarse.find(Qa + kLocalQ[s2]);
            if (cY < 0 || yoff[cY] < 0 || iL < 0 || blk_of[cY] != iL) { q.s1 = q.s0; P.push_back(q); continue; }
            const int frow = ELold.part_s_to_fine[aidx][s2];
            const Iso& U = liso_[b - 1];
            const int uk = U.out.find(Qa);
            const int dima = lb_[b].sec.dim[aidx];
            // Y is stored as (kept x rows of old L' coarse iL); op(B)[alpha][k] = Y[k, row(alpha,s2)]
            S.push_back(GemmSeg{U.mat[uk] + int64_t(EL2.f_row[f]) * dima, Y + yoff[cY] + ELold.f_row[frow],
                                dima, ycols[cY], dima, 0, 1});
          }
          q.s1 = int(S.size());
          P.push_back(q);
        }
    }
    ex_->gemm(P, S);
  }
  ex_->release(Y);
  if (psi_cur_) ex_->release(psi_cur_);
  psi_cur_ = npsi;
  psi_cur_cap_ = pn;
  tick(4);
  prepare_bond(nb);
  if (psi_n_ != pn) throw std::runtime_error("StVec: layout mismatch");
}

// ---------------------------------------------------------------------------
// sweeps

namespace {
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double unif(uint64_t& s) { return (splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }
}  // namespace

void Engine::init_sweep_state() {
  const int L = P_.L;
  // right blocks C_L .. C_2 from seeded selection isometries (kept product states),
  // with sector sizes proportional to the number of determinants of each split
  uint64_t st = P_.seed * 0x2545F4914F6CDD1Dull + 1;
  for (int m = L - 1; m >= 2; --m) {
    if (rb_[m].valid) continue;
    Enlarged E;
    E.build(rb_[m + 1].sec, false);
    auto binom = [](int n, int k) -> double {
      if (k < 0 || k > n) return 0.0;
      double r = 1;
      for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
      return r;
    };
    std::vector<QN> qs;
    std::vector<double> caps, wts;
    for (size_t c = 0; c < E.coarse.q.size(); ++c) {
      QN Q = E.coarse.q[c];
      double left = binom(m, P_.na - Q.a) * binom(m, P_.nb - Q.b);
      if (left == 0) continue;
      qs.push_back(Q);
      caps.push_back(std::min<double>(E.coarse.dim[c], left));
      wts.push_back(binom(L - m, Q.a) * binom(L - m, Q.b) * left);
    }
    // proportional split of D with caps
    std::vector<int> alloc(qs.size(), 0);
    std::vector<bool> act(qs.size(), true);
    int rem = P_.D;
    while (rem > 0) {
      double Wsum = 0;
      for (size_t k = 0; k < qs.size(); ++k)
        if (act[k]) Wsum += wts[k];
      if (Wsum <= 0) break;
      bool hit = false;
      for (size_t k = 0; k < qs.size(); ++k)
        if (act[k] && rem * wts[k] / Wsum >= caps[k] - alloc[k]) {
          rem -= int(caps[k]) - alloc[k];
          alloc[k] = int(caps[k]);
          act[k] = false;
          hit = true;
        }
      if (hit) continue;
      int used = 0;
      std::vector<std::pair<double, size_t>> fr;
      for (size_t k = 0; k < qs.size(); ++k)
        if (act[k]) {
          double sh = rem * wts[k] / Wsum;
          int f = int(std::floor(sh));
          alloc[k] += f;
          used += f;
          fr.push_back({-(sh - f), k});
        }
      std::sort(fr.begin(), fr.end());
      for (int x = 0; x < rem - used && x < int(fr.size()); ++x) alloc[fr[x].second]++;
      rem = 0;
    }
    Sectors out;
    std::vector<std::vector<double>> mats;
    for (size_t k = 0; k < qs.size(); ++k) {
      if (alloc[k] <= 0) continue;
      int c = E.coarse.find(qs[k]);
      int rows = E.coarse.dim[c];
      // choose alloc[k] distinct rows (partial Fisher-Yates)
      std::vector<int> perm(rows);
      std::iota(perm.begin(), perm.end(), 0);
      for (int x = 0; x < alloc[k]; ++x) {
        int y = x + int(splitmix(st) % uint64_t(rows - x));
        std::swap(perm[x], perm[y]);
      }
      std::vector<int> pick(perm.begin(), perm.begin() + alloc[k]);
      std::sort(pick.begin(), pick.end());
      std::vector<double> M(size_t(rows) * alloc[k], 0.0);
      for (int x = 0; x < alloc[k]; ++x) M[size_t(pick[x]) * alloc[k] + x] = 1.0;
      out.q.push_back(qs[k]);
      out.dim.push_back(alloc[k]);
      mats.push_back(std::move(M));
    }
    std::vector<const double*> mp;
    for (auto& M : mats) mp.push_back(M.data());
    load_right(m, out, mp);
  }
  build_right_blocks(2);
  prepare_bond(0);
  // random start vector
  if (psi_cur_) ex_->release(psi_cur_);
  psi_cur_ = static_cast<double*>(ex_->alloc(psi_n_ * sizeof(double)));
  psi_cur_cap_ = psi_n_;
  std::vector<double> h(psi_n_);
  for (auto& x : h) {
    double u1 = unif(st), u2 = unif(st);
    x = std::sqrt(-2.0 * std::log(u1 + 1e-300)) * std::cos(6.283185307179586 * u2);
  }
  ex_->h2d(psi_cur_, h.data(), psi_n_ * sizeof(double));
}

void Engine::tick(int k) {
  if (!timing_) return;
  phase_marks_.push_back({k, ex_->stamp()});
}

std::vector<double> Engine::run_sweeps(int nsw, const int* Dsched, double tol, int flags, int max_iter) {
  const int L = P_.L;
  if (L < 3) throw std::runtime_error("sweeps need L >= 3");
  if (!(psi_cur_ && bond_ == 0)) {
    // a loaded or swept basis (e.g. after new integrals) is rebuilt at bond 0; the
    // swept wave function is kept when its layout still fits
    if (right_buildable(2)) {
      build_right_blocks(2);
      prepare_bond(0);
    }
    if (!(psi_cur_ && bond_ == 0 && psi_cur_cap_ == psi_n_)) init_sweep_state();
  }
  std::vector<double> E;
  sweep_log_.clear();
  mode_log_.clear();
  for (double& x : phase_s) x = 0.0;
  ex_->stamps_clear();
  phase_marks_.clear();
  phase_marks_.push_back({-1, ex_->stamp()});
  timing_ = true;
  // the phase sums are taken when the sweeps end, also when a step throws
  struct PhaseSum {
    Engine* e;
    ~PhaseSum() {
      e->timing_ = false;
      try {
        for (size_t i = 1; i < e->phase_marks_.size(); ++i)
          e->phase_s[e->phase_marks_[i].first] +=
              1e-3 * e->ex_->stamp_ms(e->phase_marks_[i - 1].second, e->phase_marks_[i].second);
        e->ex_->stamps_clear();
      } catch (...) {
      }
      e->phase_marks_.clear();
    }
  } phase_sum{this};
  const bool refine_all = (flags & 1) != 0;
  for (int s = 0; s < nsw; ++s) {
    const int D = Dsched ? Dsched[s] : P_.D;
    double e = 0.0;
    int iters = 0;
    // split-BF16 sigma: FP64 residual refinement where the sweep energy is
    // reported (the last step), and at every step with refine_all; the other
    // steps stop at the split-BF16 residual floor
    auto step = [&](int b, int ltr, int refine) {
      // swap-gate layers (the brick-wall permutations of global mode optimisation):
      // even bonds on their first visit, odd bonds on the way back; the rotation by
      // pi/2 exchanges the two modes, and no eigensolver runs at that step
      const bool swap = (flags & 4) && ((b % 2 == 0) ? (ltr || b == L - 2) : !ltr);
      if (swap) {
        const double half_pi = 1.57079632679489661923;
        apply_rotation(half_pi);
        mode_log_.push_back(ModeLog{s, b, half_pi, 0.0, 0.0});
        tick(3);
        StepLog lg{s, b, ltr, e, 0, 0, 0.0, 0.0, {}};
        truncate_and_move(ltr != 0, D, &lg.discarded, &lg.kept);
        sweep_log_.push_back(std::move(lg));
        return;
      }
      e = davidson(psi_cur_, tol, max_iter, 24, &iters, refine);
      tick(1);
      if ((flags & 2) && ltr) {
        // mode optimisation micro-step: rotate the two sites' orbitals to lower the
        // entropy of the cut, the energy unchanged
        ModeLog ml{s, b, 0.0, 0.0, 0.0};
        ml.theta = mode_step(&ml.s_before, &ml.s_after);
        mode_log_.push_back(ml);
        tick(3);
      }
      StepLog lg{s, b, ltr, e, iters, last_status, last_rnorm, 0.0, {}};
      truncate_and_move(ltr != 0, D, &lg.discarded, &lg.kept);
      sweep_log_.push_back(std::move(lg));
    };
    for (int b = 0; b <= L - 3; ++b) step(b, 1, refine_all ? 1 : 0);           // left to right
    for (int b = L - 2; b >= 1; --b) step(b, 0, (refine_all || b == 1) ? 1 : 0);  // right to left
    E.push_back(e);
  }
  return E;
}

}  // namespace dmrg
