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
#include <tuple>

#include "core.h"

namespace dmrg {

namespace {

using Term = SigmaTerm;

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
  for (int& g : graph_) {
    if (g >= 0) ex_->graph_free(g);
    g = -1;
  }
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
  free_mixed();
  free_opset(EopsL_);
  free_opset(EopsR_);
  bond_ = -1;
}

void Engine::free_mixed() {
  ++plan_gen_;
  for (auto& c : mchunks_) {
    if (c.plan1 >= 0) ex_->mix_plan_free(c.plan1);
    if (c.plan2 >= 0) ex_->mix_plan_free(c.plan2);
  }
  mchunks_.clear();
  if (mplan_hl_ >= 0) ex_->mix_plan_free(mplan_hl_);
  mplan_hl_ = -1;
  if (psi_split_ >= 0) ex_->split_plan_free(psi_split_);
  psi_split_ = -1;
  for (uint16_t** p : {&oplL_, &oplR_, &oplLf_, &psiT_, &psiN_, &xpl_}) {
    if (*p) ex_->release(*p);
    *p = nullptr;
  }
  for (float** p : {&shi_, &slo_, &part_}) {
    if (*p) ex_->release(*p);
    *p = nullptr;
  }
  mixed_ready_ = false;
}

void Engine::prepare_bond(int bond) {
  const int L = P_.L;
  if (bond < 0 || bond > L - 2) throw std::runtime_error("prepare_bond: bond out of range");
  if (!lb_[bond].valid || !rb_[bond + 2].valid)
    throw std::runtime_error("prepare_bond: block operators for this bond are not built");
  free_bond();
  enlarge(true, lb_[bond], bond, EL_, EopsL_);
  enlarge(false, rb_[bond + 2], bond + 1, ER_, EopsR_);
  tick(3);
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
  tick(0);
}

std::vector<SigmaTerm> Engine::sigma_terms(bool keep_empty) const {
  const int nL = 2 * (bond_ + 1);
  const int L = P_.L;
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

  std::vector<SigmaTerm> terms;
  terms.push_back(SigmaTerm{nullptr, 0, GR(OP_H, 0), 0, 1.0});  // 1 (x) H_R'
  for (int p = 0; p < nL; ++p) {
    terms.push_back(SigmaTerm{GL(OP_C, p), 0, GR(OP_T, p), 0, 1.0});
    terms.push_back(SigmaTerm{GL(OP_C, p), 1, GR(OP_T, p), 1, -1.0});
  }
  for (int q = nL; q < 2 * L; ++q) {
    terms.push_back(SigmaTerm{GL(OP_S, q), 0, GR(OP_C, q), 1, 1.0});
    terms.push_back(SigmaTerm{GL(OP_S, q), 1, GR(OP_C, q), 0, -1.0});
  }
  for (int p = 0; p < nL; ++p)
    for (int r = p + 1; r < nL; ++r) {
      terms.push_back(SigmaTerm{GL(OP_A, p, r), 0, GR(OP_P, p, r), 0, 1.0});
      terms.push_back(SigmaTerm{GL(OP_A, p, r), 1, GR(OP_P, p, r), 1, 1.0});
    }
  for (int p = 0; p < nL; ++p)
    for (int q = p; q < nL; ++q) {
      terms.push_back(SigmaTerm{GL(OP_B, p, q), 0, GR(OP_Q, p, q), 0, 1.0});
      if (p < q) terms.push_back(SigmaTerm{GL(OP_B, p, q), 1, GR(OP_Q, p, q), 1, 1.0});
    }
  // drop terms with an empty side (the adjoint keeps them: an operator can be zero
  // for the present integrals and still have a derivative)
  std::vector<SigmaTerm> T;
  for (auto& t : terms) {
    if (!keep_empty && ((t.L && t.L->blk.empty()) || (t.R && t.R->blk.empty()))) continue;
    if (!t.L && !t.R) continue;
    T.push_back(t);
  }
  return T;
}

void Engine::build_sigma_plan() {
  ++plan_gen_;
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
  const std::vector<Term> T = sigma_terms();
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
  const int64_t xcap = P_.mem_cap ? std::max<int64_t>(int64_t(1) << 14, int64_t(P_.mem_cap / 16 / sizeof(double)))
                                  : int64_t(1) << 28;
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
  st_.n_chunks = int64_t(ranges.size());
  for (size_t i = 0; i < EL_.coarse.q.size(); ++i)
    if (psi_off_[i] >= 0) st_.max_rows = std::max<int64_t>(st_.max_rows, EL_.coarse.dim[i]);
  int64_t xmax = 0;
  for (auto& rg : ranges) {
    int64_t a = 0;
    for (size_t n = rg.first; n < rg.second; ++n) a += xsize[n];
    xmax = std::max(xmax, a);
  }
  xbuf_ = xmax ? static_cast<double*>(ex_->alloc(xmax * sizeof(double))) : nullptr;

  // fine maps of all operators used
  std::vector<FineMap> fmL(T.size()), fmR(T.size());
  host_parallel_for(int(T.size()), [&](int n) {
    fmL[n] = fine_map(T[n].L);
    fmR[n] = fine_map(T[n].R);
  });
  auto is_ident = [](const OpBlk* b) { return b->ident != 0; };
  // problems and segments are built per term (stage 1) or per output block (stage 2)
  // on host threads, then concatenated in the order a serial build gives
  struct PartPlan {
    std::vector<GemmProb> P;
    std::vector<GemmSeg> S;
    int64_t flops = 0;
  };
  auto append = [](std::vector<GemmProb>& P, std::vector<GemmSeg>& S, const PartPlan& pp) {
    const int off = int(S.size());
    for (GemmProb q : pp.P) {
      q.s0 += off;
      q.s1 += off;
      P.push_back(q);
    }
    S.insert(S.end(), pp.S.begin(), pp.S.end());
  };

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
    std::vector<PartPlan> pt(n1 - n0);
    host_parallel_for(int(n1 - n0), [&](int tn) {
      const size_t n = n0 + size_t(tn);
      PartPlan& pp = pt[size_t(tn)];
      const Term& t = T[n];
      if (!t.L) return;
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
          q.s0 = int(pp.S.size());
          for (int f : EL.coarse_fines[xb.iL]) {
            const OpBlk* ob;
            if (!t.Lt) {
              auto it = fmL[n].find({ft, f});
              if (it == fmL[n].end()) continue;
              ob = it->second;
              pp.S.push_back(GemmSeg{EopsL_.arena + ob->off, psi + int64_t(EL.f_row[f]) * cols, ob->cols,
                                   int(cols), EL.f_dim[f], 0, 0});
            } else {
              auto it = fmL[n].find({f, ft});
              if (it == fmL[n].end()) continue;
              ob = it->second;
              pp.S.push_back(GemmSeg{EopsL_.arena + ob->off, psi + int64_t(EL.f_row[f]) * cols, ob->cols,
                                   int(cols), EL.f_dim[f], 1, 0});
            }
            if (!is_ident(ob)) pp.flops += 2 * int64_t(q.M) * q.N * EL.f_dim[f];
          }
          q.s1 = int(pp.S.size());
          pp.P.push_back(q);
        }
      }
    });
    std::vector<GemmProb> P1;
    std::vector<GemmSeg> S1;
    for (const PartPlan& pp : pt) {
      append(P1, S1, pp);
      st_.flops_stage1 += pp.flops;
    }
    // ---- stage 2
    std::vector<PartPlan> pb(EL.coarse.q.size());
    host_parallel_for(int(EL.coarse.q.size()), [&](int iTi) {
      const size_t iT = size_t(iTi);
      if (psi_off_[iT] < 0) return;
      PartPlan& pp = pb[iT];
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
        q.s0 = int(pp.S.size());
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
              pp.S.push_back(GemmSeg{A + ER.f_row[g], EopsR_.arena + ob->off, int(lda), ob->cols, ER.f_dim[g], 0, 1});
            } else {
              auto it = fmR[n].find({g, gt});
              if (it == fmR[n].end()) continue;
              ob = it->second;
              pp.S.push_back(GemmSeg{A + ER.f_row[g], EopsR_.arena + ob->off, int(lda), ob->cols, ER.f_dim[g], 0, 0});
            }
            if (!is_ident(ob)) pp.flops += 2 * int64_t(q.M) * q.N * ER.f_dim[g];
          }
        }
        q.s1 = int(pp.S.size());
        pp.P.push_back(q);
      }
    });
    std::vector<GemmProb> P2;
    std::vector<GemmSeg> S2;
    for (const PartPlan& pp : pb) {
      append(P2, S2, pp);
      st_.flops_stage2 += pp.flops;
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
  // ---- split-BF16 tensor-core plans (precision 1): same terms and chunks as
  // above, evaluated on coarse (sector-level) blocks so that each stage is one
  // GEMM per block pair: stage 1 X{iT, jR} = O_L{iT <- iL} psi{iL, jR} with K =
  // the rows of iL, stage 2 sigma{iT, jT} = sum_nu X_nu{iT, jR} O_R{jT <- jR}^T
  // with K concatenated over all terms.  Fine sub-blocks that are zero stay zero
  // in the coarse operands.
  //
  // Every operand is a blocked split matrix (exec.h: rows padded to 8, K to 32,
  // three BF16 planes interleaved per 8-row group and 32-wide K slab).  Along a
  // coarse K dimension the fine sub-blocks start at multiples of 16 (rp / cp) and
  // the total is padded to 32 (rowpad / colpad), so that the padding is zero.
  if (P_.precision != 0) {
    auto pad8 = [](int64_t x) { return (x + 7) & ~int64_t(7); };
    auto pad16 = [](int64_t x) { return (x + 15) & ~int64_t(15); };
    auto pad32 = [](int64_t x) { return (x + 31) & ~int64_t(31); };
    auto bsize = [&](int64_t rows, int64_t kt) { return 3 * pad8(rows) * kt; };
    std::vector<int> rowpad(EL.coarse.q.size(), 0), colpad(ER.coarse.q.size(), 0);
    std::vector<int> rp(EL.f_dim.size(), 0), cp(ER.f_dim.size(), 0);
    for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
      for (int f : EL.coarse_fines[i]) {
        rp[f] = rowpad[i];
        rowpad[i] += int(pad16(EL.f_dim[f]));
      }
      rowpad[i] = int(pad32(rowpad[i]));
    }
    for (size_t j = 0; j < ER.coarse.q.size(); ++j) {
      for (int g : ER.coarse_fines[j]) {
        cp[g] = colpad[j];
        colpad[j] += int(pad16(ER.f_dim[g]));
      }
      colpad[j] = int(pad32(colpad[j]));
    }
    auto split_now = [&](const std::vector<SplitTask>& tk) {
      int sp = ex_->split_plan(tk);
      ex_->split_run(sp);
      ex_->split_plan_free(sp);
    };
    auto arena = [&](int64_t n) {
      uint16_t* a = static_cast<uint16_t*>(ex_->alloc(size_t(n + 64) * sizeof(uint16_t)));
      ex_->zero(a, size_t(n + 64) * sizeof(uint16_t));
      return a;
    };
    // coarse operator matrices: normal N(a <- b) is dim(a) rows x pad(b); transposed
    // T(a <- b) holds (O^T){b <- a} as dim(b) rows x pad(a).  On L' only H_L' is
    // used coarse (the local term); stage 1 reads the fine matrices below.
    using CKey = std::tuple<const Op*, int, int>;
    std::map<CKey, std::pair<int64_t, int64_t>> offL, offR;
    auto coarse = [&](const OpSet& os, const Enlarged& E, const std::vector<int>& pad, const std::vector<int>& pp,
                      const Op* only, std::map<CKey, std::pair<int64_t, int64_t>>& off, uint16_t*& ar,
                      int64_t& n) {
      int64_t o = 0;
      for (auto& kv : os.ops) {
        if (only && &kv.second != only) continue;
        for (auto& bk : kv.second.blk) {
          const int ca = E.f_coarse[bk.r], cb = E.f_coarse[bk.c];
          CKey key{&kv.second, ca, cb};
          if (off.count(key)) continue;
          const int64_t on = o;
          o += bsize(E.coarse.dim[ca], pad[cb]);
          const int64_t ot = o;
          o += bsize(E.coarse.dim[cb], pad[ca]);
          off[key] = {on, ot};
        }
      }
      n = o;
      ar = arena(n);
      std::vector<SplitTask> tk;
      for (auto& kv : os.ops) {
        if (only && &kv.second != only) continue;
        for (auto& bk : kv.second.blk) {
          const int ca = E.f_coarse[bk.r], cb = E.f_coarse[bk.c];
          const auto& oo = off[CKey{&kv.second, ca, cb}];
          tk.push_back(SplitTask{os.arena + bk.off, bk.rows, bk.cols, bk.cols, E.f_row[bk.r], pp[bk.c],
                                 int(pad8(E.coarse.dim[ca])), pad[cb], E.f_row[bk.c], pp[bk.r],
                                 int(pad8(E.coarse.dim[cb])), pad[ca], ar + oo.first, ar + oo.second});
        }
      }
      split_now(tk);
    };
    coarse(EopsL_, EL, rowpad, rp, GL(OP_H, 0), offL, oplL_, opsL_);
    coarse(EopsR_, ER, colpad, cp, nullptr, offR, oplR_, opsR_);
    // fine matrices of the L' operators for stage 1: every nonzero sub-block alone,
    // normal (rows x pad32(cols)) and transposed (cols x pad32(rows))
    {
      int64_t o = 0;
      for (auto& kv : EopsL_.ops)
        for (auto& bk : kv.second.blk) {
          bk.pn = o;
          o += bsize(bk.rows, pad32(bk.cols));
          bk.pt = o;
          o += bsize(bk.cols, pad32(bk.rows));
        }
      opsLf_ = o;
      oplLf_ = arena(o);
      std::vector<SplitTask> tk;
      for (auto& kv : EopsL_.ops)
        for (auto& bk : kv.second.blk)
          tk.push_back(SplitTask{EopsL_.arena + bk.off, bk.rows, bk.cols, bk.cols, 0, 0, int(pad8(bk.rows)),
                                 int(pad32(bk.cols)), 0, 0, int(pad8(bk.cols)), int(pad32(bk.rows)), oplLf_ + bk.pn,
                                 oplLf_ + bk.pt});
      split_now(tk);
    }
    // psi operands: psiT per fine row block f of L' (colpad(j) rows x pad32(dim f),
    // the A operand of stage 1), psiN (dim(i) rows x colpad(j)) and psiU (dim(j)
    // rows x rowpad(i)) per coarse block for the local terms
    std::vector<int64_t> tOff(EL.f_dim.size(), -1), nOff(EL.coarse.q.size(), -1), uOff(EL.coarse.q.size(), -1);
    int64_t tT = 0, tN = 0;
    for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
      if (psi_off_[i] < 0) continue;
      const int j = psi_rcoarse_[i];
      for (int f : EL.coarse_fines[i]) {
        tOff[f] = tT;
        tT += bsize(colpad[j], pad32(EL.f_dim[f]));
      }
      nOff[i] = tN;
      tN += bsize(EL.coarse.dim[i], colpad[j]);
    }
    for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
      if (psi_off_[i] < 0) continue;
      const int j = psi_rcoarse_[i];
      uOff[i] = tN;
      tN += bsize(ER.coarse.dim[j], rowpad[i]);
    }
    psT_n_ = tT;
    psN_n_ = tN;
    psiT_ = arena(tT);
    psiN_ = arena(tN);
    {
      std::vector<SplitTask> tk;
      for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
        if (psi_off_[i] < 0) continue;
        const int j = psi_rcoarse_[i];
        const int cols = ER.coarse.dim[j];
        const int dl8 = int(pad8(EL.coarse.dim[i])), dr8 = int(pad8(ER.coarse.dim[j]));
        for (int f : EL.coarse_fines[i])
          for (int g : ER.coarse_fines[j]) {
            const double* src = psi_in_ + psi_off_[i] + int64_t(EL.f_row[f]) * cols + ER.f_row[g];
            // psiN{i}: (f_row[f] + r, cp[g] + c); psiT{f}: (cp[g] + c, r);
            // psiU{i}: (f_row[g] + c, rp[f] + r)
            tk.push_back(SplitTask{src, EL.f_dim[f], ER.f_dim[g], cols, EL.f_row[f], cp[g], dl8, colpad[j],
                                   ER.f_row[g], rp[f], dr8, rowpad[i], psiN_ + nOff[i], psiN_ + uOff[i]});
            tk.push_back(SplitTask{src, EL.f_dim[f], ER.f_dim[g], cols, 0, 0, 0, 0, cp[g], 0, colpad[j],
                                   int(pad32(EL.f_dim[f])), nullptr, psiT_ + tOff[f]});
          }
      }
      psi_split_ = ex_->split_plan(tk);
    }
    // X per chunk: X{iT, jR} is dim(iT) rows x colpad(jR)
    std::vector<std::vector<int64_t>> xmoff(T.size());
    std::vector<int64_t> xmsize(T.size(), 0);
    for (size_t n = 0; n < T.size(); ++n) {
      int64_t o = 0;
      for (const XBlk& xb : xl[n]) {
        xmoff[n].push_back(o);
        o += bsize(EL.coarse.dim[xb.iT], colpad[xb.jR]);
      }
      xmsize[n] = o;
    }
    // one X buffer for all terms unless it exceeds the cap (2 bytes per element)
    const int64_t xcap_m = P_.mem_cap ? std::max<int64_t>(int64_t(3) << 14, int64_t(P_.mem_cap / 4))
                                      : int64_t(3) << 33;
    std::vector<std::pair<size_t, size_t>> mranges;
    {
      size_t st0 = 0;
      int64_t acc = 0;
      for (size_t n = 0; n < T.size(); ++n) {
        if (acc + xmsize[n] > xcap_m && n > st0) {
          mranges.push_back({st0, n});
          st0 = n;
          acc = 0;
        }
        acc += xmsize[n];
      }
      mranges.push_back({st0, T.size()});
    }
    int64_t xmax_m = 0;
    for (auto& rg : mranges) {
      int64_t a = 0;
      for (size_t n = rg.first; n < rg.second; ++n) a += xmsize[n];
      xmax_m = std::max(xmax_m, a);
    }
    xpl_n_ = xmax_m;
    st_.mix_x_elems = xmax_m / 3;
    st_.mix_plane_bytes = 2 * (opsL_ + opsR_ + opsLf_ + xpl_n_ + psT_n_ + psN_n_);
    xpl_ = arena(xpl_n_);
    shi_ = static_cast<float*>(ex_->alloc(psi_n_ * sizeof(float)));
    slo_ = static_cast<float*>(ex_->alloc(psi_n_ * sizeof(float)));
    // split-K partial sums of stage 2 (double-float pairs), reduced in a fixed
    // order, and one more slot for the local term H_L' (x) 1
    const int kMaxParts = 16;
    part_ = static_cast<float*>(ex_->alloc(size_t(kMaxParts + 1) * 2 * psi_n_ * sizeof(float)));
    ex_->zero(part_, size_t(kMaxParts + 1) * 2 * psi_n_ * sizeof(float));
    nparts_ = 1;
    for (size_t ci = 0; ci < mranges.size(); ++ci) {
      const size_t n0 = mranges[ci].first, n1 = mranges[ci].second;
      std::vector<int64_t> xb0(T.size(), 0);
      {
        int64_t a = 0;
        for (size_t n = n0; n < n1; ++n) {
          xb0[n] = a;
          a += xmsize[n];
        }
      }
      // Stage 1 on nonzero fine sub-blocks: tile rows run over rows of X, tile
      // columns over its padded R' columns.  A row block ft of X_nu that receives a
      // single fine block (ft <- f) -- every normal operator, by its Kronecker form
      // -- joins the gathered problem of (psi block, f): all such rows of all terms
      // share the B operand psi^T{jR, f} and become rows of one tall GEMM (A rows
      // and output rows from per-row tables).  Rows with several contributing f
      // (complementary S_q) are separate problems.
      // rows come in units of 8 (one 8-row group of a fine operator matrix: its
      // offset and K-slab stride); c < 0 marks a padding row past the last one.
      // Each term's rows are listed on a host thread (gathered row units with their
      // fine block f, and dense-row problems), then merged in term order.
      struct GUnit { int64_t b, bs; int64_t c[8]; float a; };
      struct TermRows {
        std::vector<std::pair<int, GUnit>> units;
        std::vector<MixProb> P;
        std::vector<MixSeg> S;
      };
      std::vector<TermRows> trows(n1 - n0);
      host_parallel_for(int(n1 - n0), [&](int tn) {
        const size_t n = n0 + size_t(tn);
        TermRows& out = trows[size_t(tn)];
        const Term& t = T[n];
        if (!t.L) return;
        for (size_t k = 0; k < xl[n].size(); ++k) {
          const XBlk& xb = xl[n][k];
          const QN qL = EL.coarse.q[xb.iL];
          const double sg = (t.R && t.R->odd && (qL.n() & 1)) ? -1.0 : 1.0;
          const int cpj = colpad[xb.jR];
          const int xr8 = int(pad8(EL.coarse.dim[xb.iT]));
          const int64_t xoff = xb0[n] + xmoff[n][k];
          for (int ft : EL.coarse_fines[xb.iT]) {
            std::vector<std::pair<int, const OpBlk*>> fs;
            for (int f : EL.coarse_fines[xb.iL]) {
              auto it = t.Lt ? fmL[n].find({f, ft}) : fmL[n].find({ft, f});
              if (it != fmL[n].end()) fs.push_back({f, it->second});
            }
            if (fs.size() == 1) {
              const int f = fs[0].first;
              const OpBlk* ob = fs[0].second;
              const int64_t b0 = t.Lt ? ob->pt : ob->pn;
              const int64_t kt = pad32(EL.f_dim[f]);
              const int br8 = int(pad8(EL.f_dim[ft]));   // rows of the fine matrix
              for (int j8 = 0; j8 < EL.f_dim[ft]; j8 += 8) {
                const int rb = j8 >> 7, hb = std::min(128, br8 - 128 * rb);
                GUnit u{b0 + int64_t(rb) * 384 * kt + ((j8 & 127) >> 3) * 768, int64_t(96) * hb, {},
                        float(t.c * sg)};
                for (int e = 0; e < 8; ++e) {
                  const int r = EL.f_row[ft] + j8 + e, xrb = r >> 7, rr = r & 127;
                  const int hx = std::min(128, xr8 - 128 * xrb);
                  u.c[e] = (j8 + e < EL.f_dim[ft])
                               ? ((xoff + int64_t(xrb) * 384 * cpj + (rr >> 3) * 768 + (rr & 7) * 8) |
                                  (int64_t(hx >> 3) << 48))
                               : -1;
                }
                out.units.push_back({f, u});
              }
              continue;
            }
            // rows with no contribution stay zero: the X buffer is cleared once when
            // all terms fit one chunk, otherwise they are written as zero problems
            if (fs.empty() && mranges.size() == 1) continue;
            MixProb q{};
            q.Cp = xpl_ + xoff;
            q.row0 = EL.f_row[ft];
            q.crows = xr8;
            q.ldc = cpj;
            q.M = EL.f_dim[ft];
            q.N = cpj;
            q.alpha = float(t.c * sg);
            q.mode = 2;
            q.cm0 = -1;
            q.s0 = int(out.S.size());
            for (auto& fb : fs) {
              const int f = fb.first;
              const uint16_t* Ap = oplLf_ + (t.Lt ? fb.second->pt : fb.second->pn);
              out.S.push_back(MixSeg{Ap, psiT_ + tOff[f], EL.f_dim[f], 0});
            }
            q.s1 = int(out.S.size());
            out.P.push_back(q);
          }
        }
      });
      std::vector<MixProb> P1;
      std::vector<MixSeg> S1;
      for (const TermRows& x : trows) {   // dense-row problems in term order
        const int off = int(S1.size());
        for (MixProb q : x.P) {
          q.s0 += off;
          q.s1 += off;
          P1.push_back(q);
        }
        S1.insert(S1.end(), x.S.begin(), x.S.end());
      }
      // one gathered problem per fine block f of L' (the psi block and its R'
      // partner follow from f), in (coarse block, f) order, rows in term order
      std::vector<int64_t> cnt(EL.f_dim.size(), 0);
      for (const TermRows& x : trows)
        for (auto& fu : x.units) ++cnt[size_t(fu.first)];
      std::vector<int> fo;
      for (size_t f = 0; f < cnt.size(); ++f)
        if (cnt[f]) fo.push_back(int(f));
      std::stable_sort(fo.begin(), fo.end(), [&](int x, int y) { return EL.f_coarse[x] < EL.f_coarse[y]; });
      std::vector<int64_t> upos(EL.f_dim.size(), 0);
      int64_t nunits = 0;
      for (int f : fo) {
        upos[size_t(f)] = nunits;
        nunits += cnt[size_t(f)];
      }
      std::vector<int64_t> bcol(size_t(2 * nunits)), ccol(size_t(8 * nunits));
      std::vector<float> acol(size_t(8 * nunits));
      for (const TermRows& x : trows)
        for (auto& fu : x.units) {
          const size_t i = size_t(upos[size_t(fu.first)]++);
          const GUnit& u = fu.second;
          bcol[2 * i] = u.b;
          bcol[2 * i + 1] = u.bs;
          for (int e = 0; e < 8; ++e) {
            ccol[8 * i + e] = u.c[e];
            acol[8 * i + e] = u.a;
          }
        }
      trows.clear();
      int64_t ubase = 0;
      for (int f : fo) {
        const int jR = psi_rcoarse_[EL.f_coarse[f]];
        MixProb q{};
        q.Cp = xpl_;
        q.ldc = colpad[jR];
        q.M = 8 * int(cnt[size_t(f)]);
        q.N = colpad[jR];
        q.alpha = 1.0f;
        q.mode = 3;
        q.cm0 = 8 * ubase;
        q.s0 = int(S1.size());
        S1.push_back(MixSeg{oplLf_, psiT_ + tOff[f], EL.f_dim[f], 0});
        q.s1 = int(S1.size());
        P1.push_back(q);
        ubase += cnt[size_t(f)];
      }
      // segments of every sigma block, then split each block's K list into parts
      struct Blk2 { int iT, jT; std::vector<MixSeg> segs; int64_t K = 0; int tiles = 0; };
      std::vector<Blk2> blks;
      for (size_t iT = 0; iT < EL.coarse.q.size(); ++iT) {
        if (psi_off_[iT] < 0) continue;
        const int jT = psi_rcoarse_[iT];
        Blk2 bk;
        bk.iT = int(iT);
        bk.jT = jT;
        for (size_t n = n0; n < n1; ++n) {
          const Term& t = T[n];
          QN dR = t.Rt ? QN{0, 0} - t.R->delta : t.R->delta;
          const int jR = rcoarse(ER.coarse.q[jT] - dR);
          if (jR < 0) continue;
          const CKey key = t.Rt ? CKey{t.R, jR, jT} : CKey{t.R, jT, jR};
          auto it = offR.find(key);
          if (it == offR.end()) continue;
          const uint16_t* B = oplR_ + (t.Rt ? it->second.second : it->second.first);
          if (!t.L) {
            if (jR != jT) continue;
            bk.segs.push_back(MixSeg{psiN_ + nOff[iT], B, colpad[jT], 0});
          } else {
            const int xi = xidx[n][iT];
            if (xi < 0 || xl[n][xi].jR != jR) continue;
            bk.segs.push_back(MixSeg{xpl_ + xb0[n] + xmoff[n][xi], B, colpad[jR], 0});
          }
          bk.K += colpad[jR];
        }
        bk.tiles = ((EL.coarse.dim[iT] + 127) / 128) * ((ER.coarse.dim[jT] + 127) / 128);
        blks.push_back(std::move(bk));
      }
      double work = 0;
      for (auto& bk : blks) work += double(bk.tiles) * double(bk.K);
      const double per_cta = std::max(1.0, work / (8.0 * 152.0));
      std::vector<MixProb> P2;
      std::vector<MixSeg> S2;
      for (auto& bk : blks) {
        int parts = int(std::ceil(double(bk.K) / per_cta));
        parts = std::max(1, std::min(kMaxParts, std::min(parts, int(bk.segs.size()))));
        nparts_ = std::max(nparts_, parts);
        size_t sidx = 0;
        int64_t done = 0;
        for (int pp = 0; pp < parts; ++pp) {
          const int64_t goal = bk.K * (pp + 1) / parts;
          MixProb q{};
          q.Chi = part_ + int64_t(pp) * 2 * psi_n_ + psi_off_[bk.iT];
          q.Clo = q.Chi + psi_n_;
          q.ldc = ER.coarse.dim[bk.jT];
          q.M = EL.coarse.dim[bk.iT];
          q.N = ER.coarse.dim[bk.jT];
          q.alpha = 1.0f;
          q.mode = 0;
          q.s0 = int(S2.size());
          while (sidx < bk.segs.size() && (done < goal || pp == parts - 1)) {
            done += bk.segs[sidx].K;
            S2.push_back(bk.segs[sidx++]);
          }
          q.s1 = int(S2.size());
          P2.push_back(q);
        }
      }
      auto count = [&](const std::vector<MixProb>& PP, const std::vector<MixSeg>& SS, int64_t& tiles, int64_t& steps) {
        for (const MixProb& q : PP) {
          int64_t st = 0;
          for (int k = q.s0; k < q.s1; ++k) st += (SS[k].K + 31) / 32;
          const int64_t t = int64_t((q.M + 127) / 128) * ((q.N + 127) / 128);
          tiles += t;
          steps += t * st;
        }
      };
      count(P1, S1, st_.mix_tiles1, st_.mix_steps1);
      count(P2, S2, st_.mix_tiles2, st_.mix_steps2);
      for (const MixProb& q : P1) (q.mode == 2 ? st_.mix_mode2 : st_.mix_mode3) += 1;
      for (const MixProb& q : P2)
        if (q.M > 128) st_.mix_multirow += 1;
      Chunk ch;
      ch.plan1 = P1.empty() ? -1 : ex_->mix_plan_g(P1, S1, bcol, ccol, acol);
      ch.plan2 = ex_->mix_plan(P2, S2);
      mchunks_.push_back(ch);
    }
    {
      const Op* HL = GL(OP_H, 0);
      std::vector<MixProb> P3;
      std::vector<MixSeg> S3;
      for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
        if (psi_off_[i] < 0) continue;
        const int j = psi_rcoarse_[i];
        auto it = offL.find(CKey{HL, int(i), int(i)});
        if (it == offL.end()) continue;
        // written into the extra part slot (never cleared: the same blocks are
        // rewritten by every call and the others stay zero)
        MixProb q{};
        q.Chi = part_ + int64_t(nparts_) * 2 * psi_n_ + psi_off_[i];
        q.Clo = q.Chi + psi_n_;
        q.ldc = ER.coarse.dim[j];
        q.M = EL.coarse.dim[i];
        q.N = ER.coarse.dim[j];
        q.alpha = 1.0f;
        q.mode = 0;
        q.s0 = int(S3.size());
        S3.push_back(MixSeg{oplL_ + it->second.first, psiN_ + uOff[i], rowpad[i], 0});
        q.s1 = int(S3.size());
        P3.push_back(q);
      }
      mplan_hl_ = P3.empty() ? -1 : ex_->mix_plan(P3, S3);
    }
    st_.mix_chunks = int64_t(mranges.size());
    st_.mix_parts = nparts_;
    mixed_ready_ = true;
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

// The kernels of one sigma step of the prepared bond, from psi_in_ to sig_out_;
// replayed from a captured CUDA graph (one per bond and precision) when the
// stream allows it, otherwise issued directly.
void Engine::sigma_body(int precision) {
  if (precision == 0 || !mixed_ready_) {
    for (auto& c : chunks_) {
      if (c.plan1 >= 0) ex_->gemm_run(c.plan1);
      ex_->gemm_run(c.plan2);
    }
    if (plan_hl_ >= 0) ex_->gemm_run(plan_hl_);
    return;
  }
  ex_->split_run(psi_split_);
  // H_L' (x) 1 goes to part slot nparts_, summed with the first chunk's parts
  if (mplan_hl_ >= 0) ex_->mix_run(mplan_hl_);
  for (size_t c = 0; c < mchunks_.size(); ++c) {
    if (mchunks_[c].plan1 >= 0) ex_->mix_run(mchunks_[c].plan1);
    ex_->zero(part_, size_t(nparts_) * 2 * psi_n_ * sizeof(float));
    ex_->mix_run(mchunks_[c].plan2);
    ex_->reduce_parts(part_, nparts_ + (c == 0 ? 1 : 0), psi_n_, shi_, slo_, c > 0);
  }
  ex_->df_to_f64(shi_, slo_, sig_out_, psi_n_);
}

void Engine::sigma_run(int precision, bool allow_capture) {
  const int k = (precision == 0 || !mixed_ready_) ? 0 : 1;
  if (allow_capture && graph_[k] < 0 && !ex_->profiling())
    graph_[k] = ex_->graph_capture([&] { sigma_body(precision); });
  if (graph_[k] >= 0 && !ex_->profiling()) {
    ex_->graph_run(graph_[k]);
    ++graph_runs_;
  } else {
    sigma_body(precision);
  }
}

void Engine::sigma(const double* psi, double* sig) {
  if (bond_ < 0) throw std::runtime_error("sigma: no bond prepared");
  ex_->d2d(psi_in_, psi, psi_n_ * sizeof(double));
  sigma_run(0);
  ex_->d2d(sig, sig_out_, psi_n_ * sizeof(double));
}

void Engine::sigma_precision(const double* psi, double* sig, int precision, bool allow_capture) {
  if (bond_ < 0) throw std::runtime_error("sigma: no bond prepared");
  ex_->d2d(psi_in_, psi, psi_n_ * sizeof(double));
  sigma_run(precision, allow_capture);
  ex_->d2d(sig, sig_out_, psi_n_ * sizeof(double));
}

void Engine::batch_prologue(const double* psi) {
  ex_->d2d(psi_in_, psi, psi_n_ * sizeof(double));
  ex_->split_run(psi_split_);
}

void Engine::batch_zero_parts() { ex_->zero(part_, size_t(nparts_) * 2 * psi_n_ * sizeof(float)); }

void Engine::batch_epilogue(double* sig) {
  // the same fixed-order reduction as the single-problem path (parts and the
  // local-term slot of the one chunk)
  ex_->reduce_parts(part_, nparts_ + 1, psi_n_, shi_, slo_, 0);
  ex_->df_to_f64(shi_, slo_, sig, psi_n_);
}

void Engine::diagonal(double* d) {
  if (bond_ < 0) throw std::runtime_error("diagonal: no bond prepared");
  ex_->d2d(d, diag_, psi_n_ * sizeof(double));
}

}  // namespace dmrg

namespace dmrg {

// Adjoint of the sigma terms (first step of integral_gradient, adjoint.cpp): for
// F = sum_terms sum_blocks < lam{iT, jT}, c s op(O_L){iT <- iL} psi{iL, jR} op(O_R){jT <- jR}^T >
// the fine blocks of every L' and R' operator listed in tl / tr receive
//   dF/d op(O_L) = c s lam op(O_R) psi^T  (via Y = c s lam op(O_R)),
//   dF/d op(O_R) = c s lam^T op(O_L) psi  (via X = c s op(O_L) psi, the stage-1 product),
// and H_L' (x) 1 gives dF/dH_L' = lam psi^T, 1 (x) H_R' gives dF/dH_R' = lam^T psi.
// Terms are processed in chunks so that X and Y stay under the memory cap; every
// adjoint block is one GEMM problem per chunk (segments summed in a fixed order,
// accumulated over the chunks in stream order).
void Engine::sigma_adjoint(const double* lam, const double* psi,
                           const std::map<OpKey, std::map<std::pair<int, int>, int64_t>>& tl, double* gl,
                           const std::map<OpKey, std::map<std::pair<int, int>, int64_t>>& tr, double* gr) {
  const Enlarged& EL = EL_;
  const Enlarged& ER = ER_;
  std::map<const Op*, OpKey> keyL, keyR;
  for (auto& kv : EopsL_.ops) keyL[&kv.second] = kv.first;
  for (auto& kv : EopsR_.ops) keyR[&kv.second] = kv.first;
  auto lcoarse = [&](const QN& q) { return EL.coarse.find(q); };
  auto rcoarse = [&](const QN& q) { return ER.coarse.find(q); };
  auto target = [](const std::map<OpKey, std::map<std::pair<int, int>, int64_t>>& tm, const OpKey& k, int r,
                   int c) -> int64_t {
    auto it = tm.find(k);
    if (it == tm.end()) return -1;
    auto jt = it->second.find({r, c});
    return jt == it->second.end() ? -1 : jt->second;
  };
  const std::vector<Term> T = sigma_terms(true);
  struct XB { int iL, jR, iT, jT; int64_t off; };
  std::vector<std::vector<XB>> xl(T.size());
  std::vector<int64_t> xsize(T.size(), 0);
  for (size_t n = 0; n < T.size(); ++n) {
    const Term& t = T[n];
    const QN dL = !t.L ? QN{0, 0} : (t.Lt ? QN{0, 0} - t.L->delta : t.L->delta);
    const QN dR = t.Rt ? QN{0, 0} - t.R->delta : t.R->delta;
    int64_t o = 0;
    for (size_t iL = 0; iL < EL.coarse.q.size(); ++iL) {
      if (psi_off_[iL] < 0) continue;
      const int jR = psi_rcoarse_[iL];
      const int iT = lcoarse(EL.coarse.q[iL] + dL);
      if (iT < 0 || psi_off_[iT] < 0) continue;
      const int jT = psi_rcoarse_[iT];
      if (rcoarse(ER.coarse.q[jR] + dR) != jT) continue;
      xl[n].push_back(XB{int(iL), jR, int(iT), jT, o});
      if (t.L) o += int64_t(EL.coarse.dim[iT]) * ER.coarse.dim[jR];
    }
    xsize[n] = o;
  }
  std::vector<FineMap> fmL(T.size()), fmR(T.size());
  for (size_t n = 0; n < T.size(); ++n) {
    fmL[n] = fine_map(T[n].L);
    fmR[n] = fine_map(T[n].R);
  }
  // chunks of terms: X and Y (each xsize) under the cap
  const int64_t cap = P_.mem_cap ? std::max<int64_t>(int64_t(1) << 14, int64_t(P_.mem_cap / 16 / sizeof(double)))
                                 : int64_t(1) << 27;
  std::vector<std::pair<size_t, size_t>> ranges;
  {
    size_t s = 0;
    int64_t acc = 0;
    for (size_t n = 0; n < T.size(); ++n) {
      if (acc + xsize[n] > cap && n > s) {
        ranges.push_back({s, n});
        s = n;
        acc = 0;
      }
      acc += xsize[n];
    }
    ranges.push_back({s, T.size()});
  }
  for (auto& rg : ranges) {
    int64_t tot = 0;
    std::vector<int64_t> base(T.size(), 0);
    for (size_t n = rg.first; n < rg.second; ++n) {
      base[n] = tot;
      tot += xsize[n];
    }
    double* X = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(tot, 1)) * sizeof(double)));
    double* Y = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(tot, 1)) * sizeof(double)));
    std::vector<GemmProb> P1;
    std::vector<GemmSeg> S1;
    // targets: C pointer -> (M, N, segments)
    struct Acc { int M, N; std::vector<GemmSeg> segs; };
    std::map<double*, Acc> acc;
    auto add = [&](double* C, int M, int N, const GemmSeg& g) {
      Acc& a = acc[C];
      a.M = M;
      a.N = N;
      a.segs.push_back(g);
    };
    for (size_t n = rg.first; n < rg.second; ++n) {
      const Term& t = T[n];
      for (const XB& xb : xl[n]) {
        const int cols = ER.coarse.dim[xb.jR], colsT = ER.coarse.dim[xb.jT], rowsT = EL.coarse.dim[xb.iT];
        const QN qL = EL.coarse.q[xb.iL];
        const double sg = (t.R && t.R->odd && (qL.n() & 1)) ? -1.0 : 1.0;
        const double* ps = psi + psi_off_[xb.iL];
        const double* lm = lam + psi_off_[xb.iT];
        const double* Xs = ps;   // identity on L': X = psi
        if (t.L) {
          double* Xb = X + base[n] + xb.off;
          double* Yb = Y + base[n] + xb.off;
          Xs = Xb;
          // X{iT, jR} = c s op(O_L) psi
          for (int ft : EL.coarse_fines[xb.iT]) {
            GemmProb q;
            q.C = Xb + int64_t(EL.f_row[ft]) * cols;
            q.ldc = cols;
            q.M = EL.f_dim[ft];
            q.N = cols;
            q.alpha = t.c * sg;
            q.accumulate = 0;
            q.s0 = int(S1.size());
            for (int f : EL.coarse_fines[xb.iL]) {
              auto it = t.Lt ? fmL[n].find({f, ft}) : fmL[n].find({ft, f});
              if (it == fmL[n].end()) continue;
              const OpBlk* ob = it->second;
              S1.push_back(GemmSeg{EopsL_.arena + ob->off, ps + int64_t(EL.f_row[f]) * cols, ob->cols, cols,
                                   EL.f_dim[f], t.Lt, 0});
            }
            q.s1 = int(S1.size());
            P1.push_back(q);
          }
          // Y{iT, jR} = c s lam{iT, jT} op(O_R){jT <- jR}
          for (int g : ER.coarse_fines[xb.jR]) {
            GemmProb q;
            q.C = Yb + ER.f_row[g];
            q.ldc = cols;
            q.M = rowsT;
            q.N = ER.f_dim[g];
            q.alpha = t.c * sg;
            q.accumulate = 0;
            q.s0 = int(S1.size());
            for (int gt : ER.coarse_fines[xb.jT]) {
              auto it = t.Rt ? fmR[n].find({g, gt}) : fmR[n].find({gt, g});
              if (it == fmR[n].end()) continue;
              const OpBlk* ob = it->second;
              S1.push_back(GemmSeg{lm + ER.f_row[gt], EopsR_.arena + ob->off, colsT, ob->cols, ER.f_dim[gt], 0, t.Rt});
            }
            q.s1 = int(S1.size());
            P1.push_back(q);
          }
          // L' operator: fine blocks (ft <- f), or (f <- ft) stored for a transposed use
          const OpKey kl = keyL.at(t.L);
          for (int ft : EL.coarse_fines[xb.iT])
            for (int f : EL.coarse_fines[xb.iL]) {
              const double* Yr = Yb + int64_t(EL.f_row[ft]) * cols;
              const double* Pr = ps + int64_t(EL.f_row[f]) * cols;
              if (!t.Lt) {
                const int64_t o = target(tl, kl, ft, f);
                if (o >= 0) add(gl + o, EL.f_dim[ft], EL.f_dim[f], GemmSeg{Yr, Pr, cols, cols, cols, 0, 1});
              } else {
                const int64_t o = target(tl, kl, f, ft);
                if (o >= 0) add(gl + o, EL.f_dim[f], EL.f_dim[ft], GemmSeg{Pr, Yr, cols, cols, cols, 0, 1});
              }
            }
        }
        // R' operator: fine blocks (gt <- g), or (g <- gt) stored for a transposed use
        const OpKey kr = keyR.at(t.R);
        for (int gt : ER.coarse_fines[xb.jT])
          for (int g : ER.coarse_fines[xb.jR]) {
            if (!t.Rt) {
              const int64_t o = target(tr, kr, gt, g);
              if (o >= 0)
                add(gr + o, ER.f_dim[gt], ER.f_dim[g], GemmSeg{lm + ER.f_row[gt], Xs + ER.f_row[g], colsT, cols, rowsT, 1, 0});
            } else {
              const int64_t o = target(tr, kr, g, gt);
              if (o >= 0)
                add(gr + o, ER.f_dim[g], ER.f_dim[gt], GemmSeg{Xs + ER.f_row[g], lm + ER.f_row[gt], cols, colsT, rowsT, 1, 0});
            }
          }
      }
    }
    if (&rg == &ranges.front()) {
      // H_L' (x) 1: dF/dH_L'{ft <- f} = lam{i}[ft rows] psi{i}[f rows]^T
      const Op* HL = EopsL_.get(OP_H, 0);
      if (HL) {
        const OpKey kh = keyL.at(HL);
        for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
          if (psi_off_[i] < 0) continue;
          const int cols = ER.coarse.dim[psi_rcoarse_[i]];
          for (int ft : EL.coarse_fines[i])
            for (int f : EL.coarse_fines[i]) {
              const int64_t o = target(tl, kh, ft, f);
              if (o < 0) continue;
              add(gl + o, EL.f_dim[ft], EL.f_dim[f],
                  GemmSeg{lam + psi_off_[i] + int64_t(EL.f_row[ft]) * cols, psi + psi_off_[i] + int64_t(EL.f_row[f]) * cols,
                          cols, cols, cols, 0, 1});
            }
        }
      }
    }
    if (!P1.empty()) ex_->gemm(P1, S1);
    std::vector<GemmProb> P2;
    std::vector<GemmSeg> S2;
    for (auto& kv : acc) {
      GemmProb q;
      q.C = kv.first;
      q.ldc = kv.second.N;
      q.M = kv.second.M;
      q.N = kv.second.N;
      q.alpha = 1.0;
      q.accumulate = 1;
      q.s0 = int(S2.size());
      S2.insert(S2.end(), kv.second.segs.begin(), kv.second.segs.end());
      q.s1 = int(S2.size());
      P2.push_back(q);
    }
    if (!P2.empty()) ex_->gemm(P2, S2);
    ex_->release(X);
    ex_->release(Y);
  }
}

}  // namespace dmrg

namespace dmrg {

// ---- term partition for sharded sigma (several GPUs, psi replicated, one sum of
// the partial sigmas): per-term work and the FP64 sigma of a subset of the terms.
// Term index nu runs over sigma_terms(); the last index is the local term
// H_L' (x) 1.

std::vector<int64_t> Engine::term_work() const {
  if (bond_ < 0) throw std::runtime_error("term_work: no bond prepared");
  const Enlarged& EL = EL_;
  const Enlarged& ER = ER_;
  const std::vector<Term> T = sigma_terms();
  std::vector<int64_t> w(T.size() + 1, 0);
  for (size_t n = 0; n < T.size(); ++n) {
    const Term& t = T[n];
    const QN dL = !t.L ? QN{0, 0} : (t.Lt ? QN{0, 0} - t.L->delta : t.L->delta);
    const QN dR = t.Rt ? QN{0, 0} - t.R->delta : t.R->delta;
    for (size_t iL = 0; iL < EL.coarse.q.size(); ++iL) {
      if (psi_off_[iL] < 0) continue;
      const int jR = psi_rcoarse_[iL];
      const int iT = EL.coarse.find(EL.coarse.q[iL] + dL);
      if (iT < 0 || psi_off_[iT] < 0) continue;
      const int jT = psi_rcoarse_[iT];
      if (ER.coarse.find(ER.coarse.q[jR] + dR) != jT) continue;
      const int64_t rows = EL.coarse.dim[iT], cols = ER.coarse.dim[jR], colsT = ER.coarse.dim[jT];
      if (t.L) w[n] += 2 * rows * cols * EL.coarse.dim[iL];
      w[n] += 2 * rows * colsT * cols;
    }
  }
  for (size_t i = 0; i < EL.coarse.q.size(); ++i)
    if (psi_off_[i] >= 0)
      w[T.size()] += 2 * int64_t(EL.coarse.dim[i]) * EL.coarse.dim[i] * ER.coarse.dim[psi_rcoarse_[i]];
  return w;
}

void Engine::sigma_subset(const double* psi, double* sig, const std::vector<char>& own) {
  if (bond_ < 0) throw std::runtime_error("sigma_subset: no bond prepared");
  const Enlarged& EL = EL_;
  const Enlarged& ER = ER_;
  const std::vector<Term> T = sigma_terms();
  if (own.size() != T.size() + 1) throw std::runtime_error("sigma_subset: owner list does not match the terms");
  ex_->zero(sig, size_t(psi_n_) * sizeof(double));
  struct XB { int iL, jR, iT, jT; int64_t off; };
  std::vector<std::vector<XB>> xl(T.size());
  std::vector<int64_t> xsize(T.size(), 0);
  for (size_t n = 0; n < T.size(); ++n) {
    if (!own[n]) continue;
    const Term& t = T[n];
    const QN dL = !t.L ? QN{0, 0} : (t.Lt ? QN{0, 0} - t.L->delta : t.L->delta);
    const QN dR = t.Rt ? QN{0, 0} - t.R->delta : t.R->delta;
    int64_t o = 0;
    for (size_t iL = 0; iL < EL.coarse.q.size(); ++iL) {
      if (psi_off_[iL] < 0) continue;
      const int jR = psi_rcoarse_[iL];
      const int iT = EL.coarse.find(EL.coarse.q[iL] + dL);
      if (iT < 0 || psi_off_[iT] < 0) continue;
      const int jT = psi_rcoarse_[iT];
      if (ER.coarse.find(ER.coarse.q[jR] + dR) != jT) continue;
      xl[n].push_back(XB{int(iL), jR, int(iT), jT, o});
      if (t.L) o += int64_t(EL.coarse.dim[iT]) * ER.coarse.dim[jR];
    }
    xsize[n] = o;
  }
  const int64_t cap = P_.mem_cap ? std::max<int64_t>(int64_t(1) << 14, int64_t(P_.mem_cap / 16 / sizeof(double)))
                                 : int64_t(1) << 28;
  std::vector<std::pair<size_t, size_t>> ranges;
  {
    size_t s = 0;
    int64_t acc = 0;
    for (size_t n = 0; n < T.size(); ++n) {
      if (acc + xsize[n] > cap && n > s) {
        ranges.push_back({s, n});
        s = n;
        acc = 0;
      }
      acc += xsize[n];
    }
    ranges.push_back({s, T.size()});
  }
  struct Sub { int M, N, ldc; std::vector<GemmSeg> segs; };
  for (auto& rg : ranges) {
    int64_t tot = 0;
    std::vector<int64_t> base(T.size(), 0);
    for (size_t n = rg.first; n < rg.second; ++n) {
      base[n] = tot;
      tot += xsize[n];
    }
    double* X = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(tot, 1)) * sizeof(double)));
    std::vector<GemmProb> P1;
    std::vector<GemmSeg> S1;
    std::map<double*, Sub> acc;   // sigma sub-block -> its segments
    for (size_t n = rg.first; n < rg.second; ++n) {
      if (!own[n]) continue;
      const Term& t = T[n];
      const FineMap fL = fine_map(t.L), fR = fine_map(t.R);
      for (const XB& xb : xl[n]) {
        const int cols = ER.coarse.dim[xb.jR], colsT = ER.coarse.dim[xb.jT], rowsT = EL.coarse.dim[xb.iT];
        const QN qL = EL.coarse.q[xb.iL];
        const double sg = (t.R && t.R->odd && (qL.n() & 1)) ? -1.0 : 1.0;
        const double* ps = psi + psi_off_[xb.iL];
        const double* Xs = ps;   // identity on L': X = psi
        if (t.L) {
          double* Xb = X + base[n] + xb.off;
          Xs = Xb;
          for (int ft : EL.coarse_fines[xb.iT]) {
            GemmProb q;
            q.C = Xb + int64_t(EL.f_row[ft]) * cols;
            q.ldc = cols;
            q.M = EL.f_dim[ft];
            q.N = cols;
            q.alpha = t.c * sg;
            q.accumulate = 0;
            q.s0 = int(S1.size());
            for (int f : EL.coarse_fines[xb.iL]) {
              auto it = t.Lt ? fL.find({f, ft}) : fL.find({ft, f});
              if (it == fL.end()) continue;
              S1.push_back(GemmSeg{EopsL_.arena + it->second->off, ps + int64_t(EL.f_row[f]) * cols, it->second->cols,
                                   cols, EL.f_dim[f], t.Lt, 0});
            }
            q.s1 = int(S1.size());
            P1.push_back(q);
          }
        }
        // sigma{iT, gt} += X{iT, jR}[:, g] op(O_R){gt <- g}^T
        for (int gt : ER.coarse_fines[xb.jT])
          for (int g : ER.coarse_fines[xb.jR]) {
            auto it = t.Rt ? fR.find({g, gt}) : fR.find({gt, g});
            if (it == fR.end()) continue;
            Sub& a = acc[sig + psi_off_[xb.iT] + ER.f_row[gt]];
            a.M = rowsT;
            a.N = ER.f_dim[gt];
            a.ldc = colsT;
            a.segs.push_back(GemmSeg{Xs + ER.f_row[g], EopsR_.arena + it->second->off, cols, it->second->cols,
                                     ER.f_dim[g], 0, t.Rt ? 0 : 1});
          }
      }
    }
    if (!P1.empty()) ex_->gemm(P1, S1);
    std::vector<GemmProb> P2;
    std::vector<GemmSeg> S2;
    for (auto& kv : acc) {
      GemmProb q;
      q.C = kv.first;
      q.M = kv.second.M;
      q.N = kv.second.N;
      q.ldc = kv.second.ldc;
      q.alpha = 1.0;
      q.accumulate = 1;
      q.s0 = int(S2.size());
      S2.insert(S2.end(), kv.second.segs.begin(), kv.second.segs.end());
      q.s1 = int(S2.size());
      P2.push_back(q);
    }
    if (!P2.empty()) ex_->gemm(P2, S2);
    ex_->release(X);
  }
  if (own[T.size()]) {
    // H_L' (x) 1
    const FineMap fm = fine_map(EopsL_.get(OP_H, 0));
    std::vector<GemmProb> P3;
    std::vector<GemmSeg> S3;
    for (size_t i = 0; i < EL.coarse.q.size(); ++i) {
      if (psi_off_[i] < 0) continue;
      const int64_t cols = ER.coarse.dim[psi_rcoarse_[i]];
      for (int ft : EL.coarse_fines[i]) {
        GemmProb q;
        q.C = sig + psi_off_[i] + int64_t(EL.f_row[ft]) * cols;
        q.ldc = int(cols);
        q.M = EL.f_dim[ft];
        q.N = int(cols);
        q.alpha = 1.0;
        q.accumulate = 1;
        q.s0 = int(S3.size());
        for (int f : EL.coarse_fines[i]) {
          auto it = fm.find({ft, f});
          if (it == fm.end()) continue;
          S3.push_back(GemmSeg{EopsL_.arena + it->second->off, psi + psi_off_[i] + int64_t(EL.f_row[f]) * cols,
                               it->second->cols, int(cols), EL.f_dim[f], 0, 0});
        }
        q.s1 = int(S3.size());
        if (q.s1 > q.s0) P3.push_back(q);
      }
    }
    if (!P3.empty()) ex_->gemm(P3, S3);
  }
}

}  // namespace dmrg
