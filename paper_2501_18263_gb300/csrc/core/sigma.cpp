// Sigma step sigma = H_eff psi at bond (k, k+1) (Eq. Hamilton_act_U1sym).
//
// With L' = B_k (x) site k and R' = site k+1 (x) C_{k+2}, normal operators on
// L' and complementary operators on R', the Hamiltonian splits as
//   H = H_L' (x) 1 + 1 (x) H_R'
//     + sum_{p in L'} (C_p T_p - C_p^T T_p^T)          (odd (x) odd)
//     + sum_{q in R'} (S_q C_q^T - S_q^T C_q)          (odd (x) odd)
//     + sum_{p<r in L'} (A_pr P_pr + A_pr^T P_pr^T)
//     + sum_{p<=q in L'} B_pq Q_pq + sum_{p<q} B_pq^T Q_pq^T
// and a product O_L O_R acts on |l>|r> with the Jordan-Wigner sign
// (-1)^{parity(O_R) * N(l)}.  Each term nu is evaluated as
//   stage 1:  X_nu{Q_L', Q_R} = c_nu sign * O_L{Q_L' <- Q_L} psi{Q_L, Q_R}
//   stage 2:  sigma{Q_L', f_R'} = sum_nu sum_{f_R} X_nu{Q_L', f_R} O_R{f_R' <- f_R}^T
// where stage 2 concatenates all (nu, f_R) along K so that the sum over terms
// happens inside one accumulator per output tile (Sec. 2.4, item (c): strided
// batched products summed without a separate reduction).  H_L' (x) 1 is added
// last as O_L psi accumulated into sigma.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "core.h"

namespace dmrg {

namespace {

struct Term {
  const Op* L;   // nullptr: identity on L'
  int Lt;
  const Op* R;   // nullptr: identity on R'
  int Rt;
  double c;
};

// fine block lookup (row fine, col fine) -> block
using FineMap = std::map<std::pair<int, int>, const OpBlk*>;

FineMap fine_map(const Op* o) {
  FineMap m;
  if (o)
    for (auto& b : o->blk) m[{b.r, b.c}] = &b;
  return m;
}

}  // namespace

void Engine::free_bond() {
  for (auto& c : chunks_) {
    if (c.plan1 >= 0) ex_->plan_free(c.plan1);
    if (c.plan2 >= 0) ex_->plan_free(c.plan2);
  }
  chunks_.clear();
  if (plan_hl_ >= 0) ex_->plan_free(plan_hl_);
  plan_hl_ = -1;
  if (diag_plan_ >= 0) ex_->plan_free(diag_plan_);
  diag_plan_ = -1;
  for (double** p : {&xbuf_, &psi_in_, &sig_out_, &diag_l_, &diag_r_, &diag_}) {
    if (*p) ex_->release(*p);
    *p = nullptr;
  }
  free_opset(EopsL_);
  free_opset(EopsR_);
  bond_ = -1;
}

void Engine::prepare_bond(int bond) {
  const int L = P_.L;
  if (bond < 0 || bond > L - 2) throw std::runtime_error("prepare_bond: bond out of range");
  if (!lb_[bond].valid || !rb_[bond + 2].valid)
    throw std::runtime_error("prepare_bond: block operators for this bond are not built");
  free_bond();
  enlarge(true, lb_[bond], bond, EL_, EopsL_);
  enlarge(false, rb_[bond + 2], bond + 1, ER_, EopsR_);
  bond_ = bond;
  // psi layout
  QN N{P_.na, P_.nb};
  lay_.clear();
  psi_off_.assign(EL_.coarse.q.size(), -1);
  psi_rcoarse_.assign(EL_.coarse.q.size(), -1);
  int64_t off = 0;
  for (size_t i = 0; i < EL_.coarse.q.size(); ++i) {
    int j = ER_.coarse.find(N - EL_.coarse.q[i]);
    if (j < 0) continue;
    psi_off_[i] = off;
    psi_rcoarse_[i] = j;
    const QN ql = EL_.coarse.q[i], qr = ER_.coarse.q[j];
    int64_t r = EL_.coarse.dim[i], c = ER_.coarse.dim[j];
    for (int64_t x : {int64_t(ql.a), int64_t(ql.b), int64_t(qr.a), int64_t(qr.b), r, c, off}) lay_.push_back(x);
    off += r * c;
  }
  psi_n_ = off;
  if (psi_n_ == 0) throw std::runtime_error("prepare_bond: empty two-site space");
  build_sigma_plan();
}

void Engine::build_sigma_plan() {
  const int L = P_.L;
  const int b = bond_;
  const int nL = 2 * (b + 1);  // spin-orbitals of L'
  st_ = BondStats();
  st_.psi_size = psi_n_;
  psi_in_ = static_cast<double*>(ex_->alloc(psi_n_ * sizeof(double)));
  sig_out_ = static_cast<double*>(ex_->alloc(psi_n_ * sizeof(double)));

  auto GL = [&](int t, int i, int j = 0) {
    const Op* o = EopsL_.get(t, i, j);
    if (!o) throw std::runtime_error("sigma plan: missing L' operator");
    return o;
  };
  auto GR = [&](int t, int i, int j = 0) {
    const Op* o = EopsR_.get(t, i, j);
    if (!o) throw std::runtime_error("sigma plan: missing R' operator");
    return o;
  };

  std::vector<Term> terms;
  terms.push_back(Term{nullptr, 0, GR(OP_H, 0), 0, 1.0});  // 1 (x) H_R'
  for (int p = 0; p < nL; ++p) {
    terms.push_back(Term{GL(OP_C, p), 0, GR(OP_T, p), 0, 1.0});
    terms.push_back(Term{GL(OP_C, p), 1, GR(OP_T, p), 1, -1.0});
  }
  for (int q = nL; q < 2 * L; ++q) {
    terms.push_back(Term{GL(OP_S, q), 0, GR(OP_C, q), 1, 1.0});
    terms.push_back(Term{GL(OP_S, q), 1, GR(OP_C, q), 0, -1.0});
  }
  for (int p = 0; p < nL; ++p)
    for (int r = p + 1; r < nL; ++r) {
      terms.push_back(Term{GL(OP_A, p, r), 0, GR(OP_P, p, r), 0, 1.0});
      terms.push_back(Term{GL(OP_A, p, r), 1, GR(OP_P, p, r), 1, 1.0});
    }
  for (int p = 0; p < nL; ++p)
    for (int q = p; q < nL; ++q) {
      terms.push_back(Term{GL(OP_B, p, q), 0, GR(OP_Q, p, q), 0, 1.0});
      if (p < q) terms.push_back(Term{GL(OP_B, p, q), 1, GR(OP_Q, p, q), 1, 1.0});
    }
  // drop terms with an empty side
  std::vector<Term> T;
  for (auto& t : terms) {
    if ((t.L && t.L->blk.empty()) || (t.R && t.R->blk.empty())) continue;
    if (!t.L && !t.R) continue;
    T.push_back(t);
  }
  st_.n_terms = int(T.size()) + 1;

  const Enlarged& EL = EL_;
  const Enlarged& ER = ER_;
  // coarse index lookups
  auto lcoarse = [&](const QN& q) { return EL.coarse.find(q); };
  auto rcoarse = [&](const QN& q) { return ER.coarse.find(q); };

  // per-term X layout: for each psi block (iL, jR) with target coarse iT
  struct XBlk { int iL, jR, iT; int64_t off; };
  std::vector<std::vector<XBlk>> xl(T.size());
  std::vector<int64_t> xsize(T.size(), 0);
  for (size_t n = 0; n < T.size(); ++n) {
    const Term& t = T[n];
    if (!t.L) continue;  // identity: X = psi
    QN dL = t.Lt ? QN{0, 0} - t.L->delta : t.L->delta;
    QN dR = t.Rt ? QN{0, 0} - t.R->delta : t.R->delta;
    int64_t o = 0;
    for (size_t iL = 0; iL < EL.coarse.q.size(); ++iL) {
      if (psi_off_[iL] < 0) continue;
      int jR = psi_rcoarse_[iL];
      int iT = lcoarse(EL.coarse.q[iL] + dL);
      if (iT < 0 || psi_off_[iT] < 0) continue;
      if (rcoarse(ER.coarse.q[jR] + dR) != psi_rcoarse_[iT]) continue;
      xl[n].push_back(XBlk{int(iL), jR, iT, o});
      o += int64_t(EL.coarse.dim[iT]) * ER.coarse.dim[jR];
    }
    xsize[n] = o;
  }
  std::vector<std::vector<int>> xidx(T.size(), std::vector<int>(EL.coarse.q.size(), -1));
  for (size_t n = 0; n < T.size(); ++n)
    for (size_t k = 0; k < xl[n].size(); ++k) xidx[n][xl[n][k].iT] = int(k);

  // chunk terms so that X fits under the scratch cap
  const int64_t xcap = std::max<int64_t>(int64_t(1) << 24, P_.mem_cap ? int64_t(P_.mem_cap / 16 / sizeof(double)) : int64_t(1) << 28);
  std::vector<std::pair<size_t, size_t>> ranges;
  {
    size_t s = 0;
    int64_t acc = 0;
    for (size_t n = 0; n < T.size(); ++n) {
      if (acc + xsize[n] > xcap && n > s) {
        ranges.push_back({s, n});
        s = n;
        acc = 0;
      }
      acc += xsize[n];
    }
    ranges.push_back({s, T.size()});
  }
  int64_t xmax = 0;
  for (auto& rg : ranges) {
    int64_t a = 0;
    for (size_t n = rg.first; n < rg.second; ++n) a += xsize[n];
    xmax = std::max(xmax, a);
  }
  xbuf_ = xmax ? static_cast<double*>(ex_->alloc(xmax * sizeof(double))) : nullptr;

  // fine maps of all operators used
  std::vector<FineMap> fmL(T.size()), fmR(T.size());
  for (size_t n = 0; n < T.size(); ++n) {
    fmL[n] = fine_map(T[n].L);
    fmR[n] = fine_map(T[n].R);
  }
  auto is_ident = [](const OpBlk* b) { return b->ident != 0; };

  for (size_t ci = 0; ci < ranges.size(); ++ci) {
    const size_t n0 = ranges[ci].first, n1 = ranges[ci].second;
    std::vector<int64_t> xbase(T.size(), 0);
    {
      int64_t a = 0;
      for (size_t n = n0; n < n1; ++n) {
        xbase[n] = a;
        a += xsize[n];
      }
    }
    // ---- stage 1
    std::vector<GemmProb> P1;
    std::vector<GemmSeg> S1;
    for (size_t n = n0; n < n1; ++n) {
      const Term& t = T[n];
      if (!t.L) continue;
      for (const XBlk& xb : xl[n]) {
        const int64_t cols = ER.coarse.dim[xb.jR];
        const QN qL = EL.coarse.q[xb.iL];
        const double sg = (t.R && t.R->odd && (qL.n() & 1)) ? -1.0 : 1.0;
        double* X = xbuf_ + xbase[n] + xb.off;
        const double* psi = psi_in_ + psi_off_[xb.iL];
        for (int ft : EL.coarse_fines[xb.iT]) {
          GemmProb q;
          q.C = X + int64_t(EL.f_row[ft]) * cols;
          q.ldc = int(cols);
          q.M = EL.f_dim[ft];
          q.N = int(cols);
          q.alpha = t.c * sg;
          q.accumulate = 0;
          q.s0 = int(S1.size());
          for (int f : EL.coarse_fines[xb.iL]) {
            const OpBlk* ob;
            if (!t.Lt) {
              auto it = fmL[n].find({ft, f});
              if (it == fmL[n].end()) continue;
              ob = it->second;
              S1.push_back(GemmSeg{EopsL_.arena + ob->off, psi + int64_t(EL.f_row[f]) * cols, ob->cols,
                                   int(cols), EL.f_dim[f], 0, 0});
            } else {
              auto it = fmL[n].find({f, ft});
              if (it == fmL[n].end()) continue;
              ob = it->second;
              S1.push_back(GemmSeg{EopsL_.arena + ob->off, psi + int64_t(EL.f_row[f]) * cols, ob->cols,
                                   int(cols), EL.f_dim[f], 1, 0});
            }
            if (!is_ident(ob)) st_.flops_stage1 += 2 * int64_t(q.M) * q.N * EL.f_dim[f];
          }
          q.s1 = int(S1.size());
          P1.push_back(q);
        }
      }
    }
    // ---- stage 2
    std::vector<GemmProb> P2;
    std::vector<GemmSeg> S2;
    for (size_t iT = 0; iT < EL.coarse.q.size(); ++iT) {
      if (psi_off_[iT] < 0) continue;
      const int jT = psi_rcoarse_[iT];
      const int64_t rows = EL.coarse.dim[iT], colsT = ER.coarse.dim[jT];
      for (int gt : ER.coarse_fines[jT]) {
        GemmProb q;
        q.C = sig_out_ + psi_off_[iT] + ER.f_row[gt];
        q.ldc = int(colsT);
        q.M = int(rows);
        q.N = ER.f_dim[gt];
        q.alpha = 1.0;
        q.accumulate = ci > 0;
        q.s0 = int(S2.size());
        for (size_t n = n0; n < n1; ++n) {
          const Term& t = T[n];
          QN dR = t.Rt ? QN{0, 0} - t.R->delta : t.R->delta;
          int jR = rcoarse(ER.coarse.q[jT] - dR);
          if (jR < 0) continue;
          const double* A;
          int64_t lda;
          if (!t.L) {
            if (jR != jT) continue;
            A = psi_in_ + psi_off_[iT];
            lda = colsT;
          } else {
            // X block (iT, jR) of term n
            const int xi = xidx[n][iT];
            if (xi < 0 || xl[n][xi].jR != jR) continue;
            const XBlk* hit = &xl[n][xi];
            A = xbuf_ + xbase[n] + hit->off;
            lda = ER.coarse.dim[jR];
          }
          for (int g : ER.coarse_fines[jR]) {
            const OpBlk* ob;
            if (!t.Rt) {
              auto it = fmR[n].find({gt, g});
              if (it == fmR[n].end()) continue;
              ob = it->second;
              S2.push_back(GemmSeg{A + ER.f_row[g], EopsR_.arena + ob->off, int(lda), ob->cols, ER.f_dim[g], 0, 1});
            } else {
              auto it = fmR[n].find({g, gt});
              if (it == fmR[n].end()) continue;
              ob = it->second;
              S2.push_back(GemmSeg{A + ER.f_row[g], EopsR_.arena + ob->off, int(lda), ob->cols, ER.f_dim[g], 0, 0});
            }
            if (!is_ident(ob)) st_.flops_stage2 += 2 * int64_t(q.M) * q.N * ER.f_dim[g];
          }
        }
        q.s1 = int(S2.size());
        P2.push_back(q);
      }
    }
    Chunk ch;
    ch.plan1 = P1.empty() ? -1 : ex_->gemm_plan(P1, S1);
    ch.plan2 = ex_->gemm_plan(P2, S2);
    st_.n_gemm_problems += int(P1.size() + P2.size());
    st_.n_gemm_segments += int(S1.size() + S2.size());
    chunks_.push_back(ch);
  }
  // ---- H_L' (x) 1, accumulated last
  {
    const Op* HL = GL(OP_H, 0);
    FineMap fm = fine_map(HL);
    std::vector<GemmProb> P3;
    std::vector<GemmSeg> S3;
    for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
      if (psi_off_[i] < 0) continue;
      const int64_t cols = ER.coarse.dim[psi_rcoarse_[i]];
      for (int ft : EL.coarse_fines[i]) {
        GemmProb q;
        q.C = sig_out_ + psi_off_[i] + int64_t(EL.f_row[ft]) * cols;
        q.ldc = int(cols);
        q.M = EL.f_dim[ft];
        q.N = int(cols);
        q.alpha = 1.0;
        q.accumulate = 1;
        q.s0 = int(S3.size());
        for (int f : EL.coarse_fines[i]) {
          auto it = fm.find({ft, f});
          if (it == fm.end()) continue;
          const OpBlk* ob = it->second;
          S3.push_back(GemmSeg{EopsL_.arena + ob->off, psi_in_ + psi_off_[i] + int64_t(EL.f_row[f]) * cols,
                               ob->cols, int(cols), EL.f_dim[f], 0, 0});
          st_.flops_stage1 += 2 * int64_t(q.M) * q.N * EL.f_dim[f];
        }
        q.s1 = int(S3.size());
        if (q.s1 > q.s0) P3.push_back(q);
      }
    }
    plan_hl_ = P3.empty() ? -1 : ex_->gemm_plan(P3, S3);
    st_.launches_per_sigma = (plan_hl_ >= 0 ? 1 : 0);
    for (auto& c : chunks_) st_.launches_per_sigma += (c.plan1 >= 0 ? 1 : 0) + 1;
    st_.n_gemm_problems += int(P3.size());
    st_.n_gemm_segments += int(S3.size());
  }
  // algorithmic operator bytes (each used operator block read once)
  {
    int64_t e = 0;
    for (auto& kv : EopsL_.ops)
      for (auto& b : kv.second.blk)
        if (!b.ident) e += int64_t(b.rows) * b.cols;
    for (auto& kv : EopsR_.ops)
      for (auto& b : kv.second.blk)
        if (!b.ident) e += int64_t(b.rows) * b.cols;
    st_.op_bytes = e * 8;
  }

  // ---- diagonal: d = dH_L (x) 1 + 1 (x) dH_R + sum_{same-spin p<=q} w_pq d(B_pq) (x) d(Q_pq)
  {
    std::vector<std::pair<const Op*, const Op*>> dt;
    std::vector<double> w;
    for (int p = 0; p < nL; ++p)
      for (int q = p; q < nL; ++q) {
        if ((p & 1) != (q & 1)) continue;
        const Op* Bo = GL(OP_B, p, q);
        const Op* Qo = GR(OP_Q, p, q);
        if (!Bo || !Qo || Bo->blk.empty() || Qo->blk.empty()) continue;
        dt.push_back({Bo, Qo});
        w.push_back(p == q ? 1.0 : 2.0);
      }
    const int nt = int(dt.size()) + 2;
    diag_l_ = static_cast<double*>(ex_->alloc(size_t(EL.coarse.total) * nt * sizeof(double)));
    diag_r_ = static_cast<double*>(ex_->alloc(size_t(ER.coarse.total) * nt * sizeof(double)));
    diag_ = static_cast<double*>(ex_->alloc(psi_n_ * sizeof(double)));
    ex_->zero(diag_l_, size_t(EL.coarse.total) * nt * sizeof(double));
    ex_->zero(diag_r_, size_t(ER.coarse.total) * nt * sizeof(double));
    diag_tasks_.clear();
    auto emit = [&](const Enlarged& E, const Op* o, double* base, int col, double coef) {
      if (!o) {  // identity column
        for (size_t f = 0; f < E.f_dim.size(); ++f) {
          int64_t row = E.coarse.off[E.f_coarse[f]] + E.f_row[f];
          diag_tasks_.push_back(DiagTask{nullptr, 0, E.f_dim[f], base + row * nt + col, nt, coef});
        }
        return;
      }
      for (auto& bk : o->blk) {
        if (bk.r != bk.c) continue;
        int64_t row = E.coarse.off[E.f_coarse[bk.r]] + E.f_row[bk.r];
        const OpBlk* p = &bk;
        const double* arena = (&E == &EL_) ? EopsL_.arena : EopsR_.arena;
        diag_tasks_.push_back(DiagTask{arena + p->off, p->cols, p->rows, base + row * nt + col, nt, coef});
      }
    };
    emit(EL, GL(OP_H, 0), diag_l_, 0, 1.0);
    emit(ER, nullptr, diag_r_, 0, 1.0);
    emit(EL, nullptr, diag_l_, 1, 1.0);
    emit(ER, GR(OP_H, 0), diag_r_, 1, 1.0);
    for (size_t k = 0; k < dt.size(); ++k) {
      emit(EL, dt[k].first, diag_l_, int(k) + 2, w[k]);
      emit(ER, dt[k].second, diag_r_, int(k) + 2, 1.0);
    }
    std::vector<GemmProb> PD;
    std::vector<GemmSeg> SD;
    for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
      if (psi_off_[i] < 0) continue;
      const int j = psi_rcoarse_[i];
      GemmProb q;
      q.C = diag_ + psi_off_[i];
      q.ldc = ER.coarse.dim[j];
      q.M = EL.coarse.dim[i];
      q.N = ER.coarse.dim[j];
      q.alpha = 1.0;
      q.accumulate = 0;
      q.s0 = int(SD.size());
      SD.push_back(GemmSeg{diag_l_ + EL.coarse.off[i] * nt, diag_r_ + ER.coarse.off[j] * nt, nt, nt, nt, 0, 1});
      q.s1 = int(SD.size());
      PD.push_back(q);
    }
    ex_->diag(diag_tasks_);
    diag_plan_ = ex_->gemm_plan(PD, SD);
    ex_->gemm_run(diag_plan_);
  }
}

void Engine::sigma(const double* psi, double* sig) {
  if (bond_ < 0) throw std::runtime_error("sigma: no bond prepared");
  ex_->d2d(psi_in_, psi, psi_n_ * sizeof(double));
  for (auto& c : chunks_) {
    if (c.plan1 >= 0) ex_->gemm_run(c.plan1);
    ex_->gemm_run(c.plan2);
  }
  if (plan_hl_ >= 0) ex_->gemm_run(plan_hl_);
  ex_->d2d(sig, sig_out_, psi_n_ * sizeof(double));
}

void Engine::sigma_precision(const double* psi, double* sig, int precision) {
  (void)precision;
  sigma(psi, sig);
}

void Engine::rdm(const double* lam, const double* psi, double* g1, double* g2) {
  (void)lam; (void)psi; (void)g1; (void)g2;
  throw std::runtime_error("dmrg_sigma_backward: not available in this build");
}

void Engine::diagonal(double* d) {
  if (bond_ < 0) throw std::runtime_error("diagonal: no bond prepared");
  ex_->d2d(d, diag_, psi_n_ * sizeof(double));
}

}  // namespace dmrg
