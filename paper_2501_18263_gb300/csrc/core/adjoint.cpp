// Adjoint of the operator construction: the derivatives of
//     F = <lam| H_eff(t, v) |psi>
// with respect to the integrals t and v for a fixed MPS basis.  For lam = psi the
// normalised ground state, dF/dt_ij is the one-particle density matrix and dF/dv_ijkl
// half the two-particle one (the differentiation form; Sec. 2.2 needs these densities
// for the orbital rotations c~+ = U c+ of mode optimisation).
//
// F depends on the integrals only through the coefficients of the blocking steps
// (site matrices and integral-weighted sums of block operators, Sec. 2.3) and is
// linear in them.  Reverse mode:
//   1. at the bond, the adjoint of every fine block of every L' and R' operator from
//      the sigma terms (sigma_adjoint, sigma.cpp): for a term c op(O_L) (x) op(O_R)
//      and a psi block,  dF/dO_L = c s lam O_R psi^T  and  dF/dO_R = c s lam^T O_L psi
//      (s the Jordan-Wigner sign of the block);
//   2. down the left chain (B_b (x) site b, B_{b-1} (x) site b-1, ..., B_0 (x) site 0)
//      and up the right chain (site b+1 (x) C_{b+2}, ..., site L-1 (x) C_L): for each
//      blocking contribution E{rf, cf} += coef * op(src),
//        adj(src) += coef * op^T(adj E{rf, cf})      (a Kronecker accumulation)
//        dF/dcoef  = <adj E{rf, cf}, op(src)>        (a Frobenius product)
//      and dF/dcoef is spread over the integrals of coef (a linear form); then through
//      the renormalisation B' = U^T E U that made the block:
//        adj E{fr, fc} = U{fr rows} adj B'{r, c} U{fc rows}^T.
// The forward operators are the ones the engine already holds for the bond; the
// adjoint keeps one block's and one enlarged block's adjoints at a time, and cuts the
// sigma-term intermediates into chunks under mem_cap.
#include <algorithm>
#include <map>
#include <stdexcept>

#include "core.h"

namespace dmrg {

namespace {

using TargetMap = std::map<OpKey, std::map<std::pair<int, int>, int64_t>>;

// one blocking step: its contributions and the fine blocks whose adjoints it reads
struct AdjStep {
  Enlarged E;
  std::vector<BlockingTerm> bt;
  TargetMap tgt;   // (operator, fine block) -> offset in the step's adjoint arena
  int64_t n = 0;
};

}  // namespace

namespace {

AdjStep make_step(const Engine& eng, bool left, const Block& blk, int site) {
  AdjStep s;
  s.bt = eng.blocking_terms(left, blk, site, s.E);
  for (const BlockingTerm& x : s.bt) {
    auto& m = s.tgt[x.key];
    auto it = m.find({x.rf, x.cf});
    if (it != m.end()) continue;
    m[{x.rf, x.cf}] = s.n;
    s.n += int64_t(s.E.f_dim[x.rf]) * s.E.f_dim[x.cf];
  }
  return s;
}

}  // namespace

void Engine::set_integrals(const std::vector<double>& t, const std::vector<double>& v) {
  const size_t L2 = size_t(P_.L) * P_.L;
  if (t.size() != L2 || v.size() != L2 * L2) throw std::runtime_error("set_integrals: wrong sizes");
  free_bond();
  P_.t = t;
  P_.v = v;
  for (int n = 1; n <= P_.L; ++n) {
    free_opset(lb_[n].ops);
    lb_[n].valid = false;
  }
  for (int m = 0; m < P_.L; ++m) {
    free_opset(rb_[m].ops);
    rb_[m].valid = false;
  }
}

void Engine::integral_gradient(const double* lam, const double* psi, std::vector<double>& raw) {
  if (bond_ < 0) throw std::runtime_error("integral_gradient: no bond prepared");
  const int L = P_.L, b = bond_;
  const int64_t L2 = int64_t(L) * L;
  raw.assign(size_t(L2 + L2 * L2), 0.0);
  if (!lb_[b].valid || !rb_[b + 2].valid) throw std::runtime_error("integral_gradient: blocks not built");

  // Frobenius products of the adjoints with the operators they multiply, spread over
  // the integrals of each coefficient (host, in a fixed order)
  auto spread = [&](const std::vector<DotTask>& dt, const std::vector<const Lin*>& dl) {
    if (dt.empty()) return;
    double* d = static_cast<double*>(ex_->alloc(dt.size() * sizeof(double)));
    ex_->dots(dt, d);
    std::vector<double> h(dt.size());
    ex_->d2h(h.data(), d, h.size() * sizeof(double));
    ex_->release(d);
    for (size_t i = 0; i < h.size(); ++i)
      for (const auto& w : dl[i]->w) raw[size_t(w.first)] += w.second * h[i];
  };

  // blocking step backwards: adjoint of the block operators (arena of blk.ops's
  // layout, allocated here) and the coefficient derivatives
  auto back_blocking = [&](const AdjStep& st, const Block& blk, const double* adjE) -> double* {
    const int64_t nb = std::max<int64_t>(blk.ops.n_elem, 1);
    double* ob = static_cast<double*>(ex_->alloc(size_t(nb) * sizeof(double)));
    ex_->zero(ob, size_t(nb) * sizeof(double));
    std::map<std::pair<const Op*, int>, std::vector<KronTask>> groups;
    std::vector<DotTask> dt;
    std::vector<const Lin*> dl;
    for (const BlockingTerm& x : st.bt) {
      const int64_t go = st.tgt.at(x.key).at({x.rf, x.cf});
      const int rows = st.E.f_dim[x.rf], cols = st.E.f_dim[x.cf];
      const double* g = adjE + go;
      if (x.src) {
        const double val = lin_value(x.coef);
        if (val != 0.0) groups[{x.src, x.src_blk}].push_back(KronTask{g, cols, x.trans, val});
      }
      if (!x.coef.w.empty()) {
        if (x.src) {
          const OpBlk& sb = x.src->blk[x.src_blk];
          dt.push_back(DotTask{g, blk.ops.arena + sb.off, cols, sb.cols, rows, cols, x.trans});
        } else {
          dt.push_back(DotTask{g, nullptr, cols, 0, rows, cols, 2});
        }
        dl.push_back(&x.coef);
      }
    }
    std::vector<KronGroup> kg;
    std::vector<KronTask> kt;
    for (auto& gv : groups) {
      const OpBlk& sb = gv.first.first->blk[gv.first.second];
      KronGroup g;
      g.dst = ob + sb.off;
      g.ld = sb.cols;
      g.rows = sb.rows;
      g.cols = sb.cols;
      g.t0 = int(kt.size());
      g.accumulate = 0;
      kt.insert(kt.end(), gv.second.begin(), gv.second.end());
      g.t1 = int(kt.size());
      kg.push_back(g);
    }
    if (!kg.empty()) ex_->kron(kg, kt);
    spread(dt, dl);
    return ob;
  };

  // renormalisation backwards: adjoint of the enlarged block of step `nx` (whose
  // isometry `iso` made block `B`) from the adjoint `ob` of B's operators
  auto back_renorm = [&](const AdjStep& nx, const Iso& iso, const Block& B, const double* ob) -> double* {
    const int64_t ne = std::max<int64_t>(nx.n, 1);
    double* ge = static_cast<double*>(ex_->alloc(size_t(ne) * sizeof(double)));
    ex_->zero(ge, size_t(ne) * sizeof(double));
    const Enlarged& E = nx.E;
    std::vector<int> c2s(E.coarse.q.size(), -1);
    for (size_t k = 0; k < iso.out.q.size(); ++k) {
      const int c = E.coarse.find(iso.out.q[k]);
      if (c < 0 || E.coarse.dim[c] != iso.rows[k]) throw std::runtime_error("adjoint: isometry and enlarged basis differ");
      c2s[c] = int(k);
    }
    // W(op, block) = adj B'{r <- c} U_c^T (dr x rows_c), then adj E{fr, fc} = U_r{fr rows} W{fc cols}
    struct Need { const Op* op; int bi; std::vector<std::pair<int64_t, std::pair<int, int>>> t; };
    std::map<std::pair<const Op*, int>, Need> need;
    for (auto& kv : nx.tgt) {
      auto oit = B.ops.ops.find(kv.first);
      if (oit == B.ops.ops.end()) continue;
      const Op& bo = oit->second;
      for (auto& tv : kv.second) {
        const int rf = tv.first.first, cf = tv.first.second;
        const int r = c2s[E.f_coarse[rf]], c = c2s[E.f_coarse[cf]];
        if (r < 0 || c < 0) continue;
        auto bit = bo.by_col.find(c);
        if (bit == bo.by_col.end() || bo.blk[bit->second].r != r) continue;
        Need& nd = need[{&bo, bit->second}];
        nd.op = &bo;
        nd.bi = bit->second;
        nd.t.push_back({tv.second, {rf, cf}});
      }
    }
    const int64_t cap = int64_t(1) << 27;
    double* W = nullptr;
    int64_t wcap = 0;
    std::vector<GemmProb> p1, p2;
    std::vector<GemmSeg> s1, s2;
    int64_t used = 0;
    auto flush = [&]() {
      if (!p1.empty()) ex_->gemm(p1, s1);
      if (!p2.empty()) ex_->gemm(p2, s2);
      p1.clear(); p2.clear(); s1.clear(); s2.clear();
      used = 0;
    };
    for (auto& nv : need) {
      const Need& nd = nv.second;
      const OpBlk& bk = nd.op->blk[nd.bi];
      const int r = bk.r, c = bk.c;
      const int dr = iso.out.dim[r], dc = iso.out.dim[c], rows_c = iso.rows[c];
      const int64_t sz = int64_t(dr) * rows_c;
      if (used + sz > wcap) {
        flush();
        if (sz > wcap) {
          if (W) ex_->release(W);
          wcap = std::max(sz, std::min(cap, int64_t(1) << 22));
          W = static_cast<double*>(ex_->alloc(size_t(wcap) * sizeof(double)));
        }
      }
      double* w = W + used;
      used += sz;
      GemmProb q;
      q.C = w;
      q.ldc = rows_c;
      q.M = dr;
      q.N = rows_c;
      q.alpha = 1.0;
      q.accumulate = 0;
      q.s0 = int(s1.size());
      s1.push_back(GemmSeg{ob + bk.off, iso.mat[c], dc, dc, dc, 0, 1});
      q.s1 = int(s1.size());
      p1.push_back(q);
      for (auto& tg : nd.t) {
        const int rf = tg.second.first, cf = tg.second.second;
        GemmProb q2;
        q2.C = ge + tg.first;
        q2.ldc = E.f_dim[cf];
        q2.M = E.f_dim[rf];
        q2.N = E.f_dim[cf];
        q2.alpha = 1.0;
        q2.accumulate = 0;
        q2.s0 = int(s2.size());
        s2.push_back(GemmSeg{iso.mat[r] + int64_t(E.f_row[rf]) * dr, w + E.f_row[cf], dr, rows_c, dr, 0, 0});
        q2.s1 = int(s2.size());
        p2.push_back(q2);
      }
    }
    flush();
    if (W) ex_->release(W);
    return ge;
  };

  // 1. the bond
  AdjStep SL = make_step(*this, true, lb_[b], b);
  AdjStep SR = make_step(*this, false, rb_[b + 2], b + 1);
  double* gl = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(SL.n, 1)) * sizeof(double)));
  double* gr = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(SR.n, 1)) * sizeof(double)));
  ex_->zero(gl, size_t(std::max<int64_t>(SL.n, 1)) * sizeof(double));
  ex_->zero(gr, size_t(std::max<int64_t>(SR.n, 1)) * sizeof(double));
  sigma_adjoint(lam, psi, SL.tgt, gl, SR.tgt, gr);

  // 2. left chain: step n enlarges B_n with site n; B_n came from step n-1
  {
    AdjStep cur = std::move(SL);
    double* adj = gl;
    for (int n = b; n >= 0; --n) {
      double* ob = back_blocking(cur, lb_[n], adj);
      ex_->release(adj);
      if (n == 0) {
        ex_->release(ob);
        break;
      }
      AdjStep nx = make_step(*this, true, lb_[n - 1], n - 1);
      adj = back_renorm(nx, liso_[n - 1], lb_[n], ob);
      ex_->release(ob);
      cur = std::move(nx);
    }
  }
  // right chain: step m enlarges C_{m+1} with site m; C_{m+1} came from step m+1
  {
    AdjStep cur = std::move(SR);
    double* adj = gr;
    for (int m = b + 1; m <= L - 1; ++m) {
      double* ob = back_blocking(cur, rb_[m + 1], adj);
      ex_->release(adj);
      if (m == L - 1) {
        ex_->release(ob);
        break;
      }
      AdjStep nx = make_step(*this, false, rb_[m + 2], m + 1);
      adj = back_renorm(nx, riso_[m + 1], rb_[m + 1], ob);
      ex_->release(ob);
      cur = std::move(nx);
    }
  }
  ex_->sync();
}

}  // namespace dmrg
