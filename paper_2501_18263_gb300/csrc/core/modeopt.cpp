// Mode optimisation micro-step (Sec. 2.2, Fig. 1): at bond (k, k+1), after the
// eigenstate Psi is found, search the two-site orbital rotation u^(k,k+1) that
// minimises the half-Renyi block entropy S_1/2 = 2 ln Tr sqrt(rho) of the cut
// between sites k and k+1, then rotate Psi and the integrals t, v with it so that
// the Hamiltonian (and the energy) stays the same.
//
// The rotation is spin independent: with c = cos(theta), s = sin(theta), the new
// orbitals are  c~+_{k,s} = c c+_{k,s} + s c+_{k+1,s},  c~+_{k+1,s} = -s c+_{k,s} + c c+_{k+1,s}
// (U = [[c, s], [-s, c]] on positions k, k+1), so t -> U t U^T and every index of v
// rotates alike.  On the 16 states of the two sites (local states 0, beta, alpha,
// alpha beta, Jordan-Wigner order site k before site k+1, alpha before beta) the
// coefficients in the new orbitals are C'(n') = sum_n <n'|n> C(n); the overlaps
// are built from the creation operators themselves, so the fermionic signs follow
// from the operator algebra.  Rotations by +-pi/2 exchange the two modes (a swap
// gate, with a sign on the second one).
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "core.h"

namespace dmrg {

namespace {

// 16 x 16 matrices on the two-site space, index 4 s1 + s2
struct M16 {
  double a[16][16] = {};
};

M16 mul(const M16& x, const M16& y) {
  M16 r;
  for (int i = 0; i < 16; ++i)
    for (int k = 0; k < 16; ++k) {
      if (x.a[i][k] == 0.0) continue;
      for (int j = 0; j < 16; ++j) r.a[i][j] += x.a[i][k] * y.a[k][j];
    }
  return r;
}

M16 lin(double p, const M16& x, double q, const M16& y) {
  M16 r;
  for (int i = 0; i < 16; ++i)
    for (int j = 0; j < 16; ++j) r.a[i][j] = p * x.a[i][j] + q * y.a[i][j];
  return r;
}

// creation operator of spin sigma on site `which` (0: k, 1: k+1) of the pair
M16 cdag2(int which, int sigma) {
  const Site4 c = site_cdag(sigma);
  static const double par[4] = {1.0, -1.0, -1.0, 1.0};   // (-1)^N of one site
  M16 r;
  for (int s1 = 0; s1 < 4; ++s1)
    for (int s2 = 0; s2 < 4; ++s2)
      for (int t1 = 0; t1 < 4; ++t1)
        for (int t2 = 0; t2 < 4; ++t2) {
          double v;
          if (which == 0) v = (s2 == t2) ? c.m[s1][t1] : 0.0;
          else v = (s1 == t1) ? par[s1] * c.m[s2][t2] : 0.0;
          r.a[4 * s1 + s2][4 * t1 + t2] = v;
        }
  return r;
}

}  // namespace

// W[n][n'] = <n | n'~>: column n' is the new-orbital basis state n' in the old basis
std::vector<double> two_site_rotation(double theta) {
  const double c = std::cos(theta), s = std::sin(theta);
  M16 cd[2][2], nd[2][2];
  for (int w = 0; w < 2; ++w)
    for (int sg = 0; sg < 2; ++sg) cd[w][sg] = cdag2(w, sg);
  for (int sg = 0; sg < 2; ++sg) {
    nd[0][sg] = lin(c, cd[0][sg], s, cd[1][sg]);
    nd[1][sg] = lin(-s, cd[0][sg], c, cd[1][sg]);
  }
  M16 id;
  for (int i = 0; i < 16; ++i) id.a[i][i] = 1.0;
  // the operator that creates local state t of one site from nothing: 0 -> 1,
  // beta -> c+_b, alpha -> c+_a, alpha beta -> c+_a c+_b
  auto make = [&](const M16* op, int t) {
    if (t == 0) return id;
    if (t == 1) return op[1];
    if (t == 2) return op[0];
    return mul(op[0], op[1]);
  };
  std::vector<double> W(256, 0.0);
  for (int t1 = 0; t1 < 4; ++t1)
    for (int t2 = 0; t2 < 4; ++t2) {
      const M16 o = mul(make(nd[0], t1), make(nd[1], t2));
      for (int n = 0; n < 16; ++n) W[n * 16 + (4 * t1 + t2)] = o.a[n][0];   // applied to |0, 0>
    }
  return W;
}

void Engine::rotate_two_site(double theta, const double* in, double* out) {
  if (bond_ < 0) throw std::runtime_error("rotate_two_site: no bond prepared");
  const std::vector<double> W = two_site_rotation(theta);
  const Enlarged& EL = EL_;
  const Enlarged& ER = ER_;
  // psi'[(l, s1'), (s2', r)] = sum_{s1, s2} <s1' s2'~ | s1 s2> psi[(l, s1), (s2, r)]  (<n'~|n> = W[n][n'])
  std::vector<KronGroup> g;
  std::vector<KronTask> tk;
  const Sectors& BL = lb_[bond_].sec;
  const Sectors& CR = rb_[bond_ + 2].sec;
  for (size_t kl = 0; kl < BL.q.size(); ++kl)
    for (size_t kr = 0; kr < CR.q.size(); ++kr)
      for (int a1 = 0; a1 < 4; ++a1)
        for (int a2 = 0; a2 < 4; ++a2) {
          const int fL = EL.part_s_to_fine[kl][a1], fR = ER.part_s_to_fine[kr][a2];
          if (fL < 0 || fR < 0) continue;
          const int iL = EL.f_coarse[fL];
          if (psi_off_[iL] < 0 || psi_rcoarse_[iL] != ER.f_coarse[fR]) continue;
          const int cols = ER.coarse.dim[psi_rcoarse_[iL]];
          KronGroup kg;
          kg.dst = out + psi_off_[iL] + int64_t(EL.f_row[fL]) * cols + ER.f_row[fR];
          kg.ld = cols;
          kg.rows = EL.f_dim[fL];
          kg.cols = ER.f_dim[fR];
          kg.accumulate = 0;
          kg.t0 = int(tk.size());
          for (int b1 = 0; b1 < 4; ++b1)
            for (int b2 = 0; b2 < 4; ++b2) {
              const double w = W[(4 * b1 + b2) * 16 + (4 * a1 + a2)];
              if (w == 0.0) continue;
              const int gL = EL.part_s_to_fine[kl][b1], gR = ER.part_s_to_fine[kr][b2];
              if (gL < 0 || gR < 0) continue;
              const int jL = EL.f_coarse[gL];
              if (psi_off_[jL] < 0 || psi_rcoarse_[jL] != ER.f_coarse[gR]) continue;
              const int cs = ER.coarse.dim[psi_rcoarse_[jL]];
              tk.push_back(KronTask{in + psi_off_[jL] + int64_t(EL.f_row[gL]) * cs + ER.f_row[gR], cs, 0, w});
            }
          kg.t1 = int(tk.size());
          g.push_back(kg);
        }
  if (in == out) throw std::runtime_error("rotate_two_site: in and out must differ");
  ex_->zero(out, size_t(psi_n_) * sizeof(double));
  if (!g.empty()) ex_->kron(g, tk);
}

std::vector<double> Engine::left_spectrum(const double* psi) {
  if (bond_ < 0) throw std::runtime_error("left_spectrum: no bond prepared");
  // the nonzero eigenvalues of rho = psi psi^T are those of the smaller Gram matrix of
  // each psi block (psi psi^T or psi^T psi): no structural zeros, whose rounding would
  // otherwise add about sqrt(eps) each to Tr sqrt(rho)
  std::vector<int> blk, dims;
  std::vector<int64_t> roff;
  int64_t tot = 0, totw = 0;
  for (size_t i = 0; i < EL_.coarse.q.size(); ++i) {
    if (psi_off_[i] < 0) continue;
    const int g = std::min(EL_.coarse.dim[i], ER_.coarse.dim[psi_rcoarse_[i]]);
    blk.push_back(int(i));
    dims.push_back(g);
    roff.push_back(tot);
    tot += int64_t(g) * g;
    totw += g;
  }
  double* rho = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(tot, 1)) * sizeof(double)));
  double* Z = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(tot, 1)) * sizeof(double)));
  double* wv = static_cast<double*>(ex_->alloc(size_t(std::max<int64_t>(totw, 1)) * sizeof(double)));
  std::vector<GemmProb> P;
  std::vector<GemmSeg> S;
  for (size_t k = 0; k < blk.size(); ++k) {
    const int i = blk[k];
    const int rows = EL_.coarse.dim[i], cols = ER_.coarse.dim[psi_rcoarse_[i]];
    GemmProb q;
    q.C = rho + roff[k];
    q.ldc = dims[k];
    q.M = dims[k];
    q.N = dims[k];
    q.alpha = 1.0;
    q.accumulate = 0;
    q.s0 = int(S.size());
    if (rows <= cols) S.push_back(GemmSeg{psi + psi_off_[i], psi + psi_off_[i], cols, cols, cols, 0, 1});   // psi psi^T
    else S.push_back(GemmSeg{psi + psi_off_[i], psi + psi_off_[i], cols, cols, rows, 1, 0});                // psi^T psi
    q.s1 = int(S.size());
    P.push_back(q);
  }
  ex_->gemm(P, S);
  std::vector<double*> Av, wvv, Zv;
  int64_t wo = 0;
  for (size_t k = 0; k < blk.size(); ++k) {
    Av.push_back(rho + roff[k]);
    Zv.push_back(Z + roff[k]);
    wvv.push_back(wv + wo);
    wo += dims[k];
  }
  ex_->syev(Av, wvv, Zv, dims);
  std::vector<double> w(static_cast<size_t>(totw));
  ex_->d2h(w.data(), wv, size_t(totw) * sizeof(double));
  for (double* p : {rho, Z, wv}) ex_->release(p);
  return w;
}

double Engine::half_renyi(const double* psi) {
  const std::vector<double> w = left_spectrum(psi);
  double s = 0.0, n = 0.0;
  for (double x : w) {
    s += std::sqrt(std::max(0.0, x));
    n += std::max(0.0, x);
  }
  // normalised state: Tr rho = 1
  return n > 0 ? 2.0 * std::log(s / std::sqrt(n)) : 0.0;
}

double Engine::entropy_at(double theta, const double* psi, double* scratch) {
  rotate_two_site(theta, psi, scratch);
  return half_renyi(scratch);
}

double Engine::best_rotation(const double* psi, double* s_min, double* s0_out) {
  if (bond_ < 0) throw std::runtime_error("best_rotation: no bond prepared");
  double* tmp = static_cast<double*>(ex_->alloc(size_t(psi_n_) * sizeof(double)));
  const double pi = 3.14159265358979323846;
  // coarse scan of one period of the entropy (rotations by pi exchange signs only),
  // then golden-section refinement around the best grid point
  const int ng = 24;
  std::vector<double> th(ng), sv(ng);
  for (int i = 0; i < ng; ++i) {
    th[i] = -pi / 2 + pi * i / ng;
    sv[i] = entropy_at(th[i], psi, tmp);
  }
  const double s0 = half_renyi(psi);
  int ib = int(std::min_element(sv.begin(), sv.end()) - sv.begin());
  double a = th[ib] - pi / ng, b = th[ib] + pi / ng;
  const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
  double f1 = entropy_at(x1, psi, tmp), f2 = entropy_at(x2, psi, tmp);
  for (int it = 0; it < 30 && b - a > 1e-9; ++it) {
    if (f1 < f2) {
      b = x2;
      x2 = x1;
      f2 = f1;
      x1 = b - gr * (b - a);
      f1 = entropy_at(x1, psi, tmp);
    } else {
      a = x1;
      x1 = x2;
      f1 = f2;
      x2 = a + gr * (b - a);
      f2 = entropy_at(x2, psi, tmp);
    }
  }
  double best = f1 < f2 ? x1 : x2, sb = std::min(f1, f2);
  if (!(sb < s0)) {   // no rotation lowers the entropy
    best = 0.0;
    sb = s0;
  }
  ex_->release(tmp);
  if (s_min) *s_min = sb;
  if (s0_out) *s0_out = s0;
  return best;
}

void Engine::rotate_integrals_pair(int k, double theta, bool rebuild) {
  const int L = P_.L;
  const double c = std::cos(theta), s = std::sin(theta);
  // U = identity except U[k][k] = c, U[k][k+1] = s, U[k+1][k] = -s, U[k+1][k+1] = c
  auto Ur = [&](int a, int i) -> double {
    if (a != k && a != k + 1) return a == i ? 1.0 : 0.0;
    if (i != k && i != k + 1) return 0.0;
    if (a == k) return i == k ? c : s;
    return i == k ? -s : c;
  };
  const size_t L2 = size_t(L) * L;
  std::vector<double> t2(L2, 0.0), v1(L2 * L2, 0.0), v2(L2 * L2, 0.0);
  // t' = U t U^T
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b) {
      double x = 0.0;
      for (int i = 0; i < L; ++i) {
        const double ua = Ur(a, i);
        if (ua == 0.0) continue;
        for (int j = 0; j < L; ++j) {
          const double ub = Ur(b, j);
          if (ub != 0.0) x += ua * ub * P_.t[size_t(i) * L + j];
        }
      }
      t2[size_t(a) * L + b] = x;
    }
  // v'_abcd = sum U_ai U_bj U_ck U_dl v_ijkl, one index at a time
  std::vector<double> cur = P_.v;
  for (int ax = 0; ax < 4; ++ax) {
    std::vector<double>& nx = (ax % 2 == 0) ? v1 : v2;
    std::fill(nx.begin(), nx.end(), 0.0);
    for (size_t e = 0; e < cur.size(); ++e) {
      const double x = cur[e];
      if (x == 0.0) continue;
      size_t idx[4] = {e / (L2 * L), (e / L2) % L, (e / L) % L, e % L};
      const int i = int(idx[ax]);
      for (int a = 0; a < L; ++a) {
        const double u = Ur(a, i);
        if (u == 0.0) continue;
        size_t id2[4] = {idx[0], idx[1], idx[2], idx[3]};
        id2[ax] = size_t(a);
        nx[((id2[0] * L + id2[1]) * L + id2[2]) * L + id2[3]] += u * x;
      }
    }
    cur = nx;
  }
  if (rebuild) {
    set_integrals(t2, cur);
  } else {
    P_.t = t2;
    P_.v = cur;
  }
}

// The stored block operators after the rotation of the orbitals at chain positions
// k, k+1 (both explicit at bond k).  No block holds those orbitals inside it; they
// enter only as the external indices of complementary operators, each of which is
// linear in every external index:  S_q on left blocks,  T_p, P_pr, Q_pq on right
// blocks.  So  O'_{x..} = sum_y U_xy O_{y..}  per rotated index (U acting on the
// spatial orbital, spin kept), with P_rp = -P_pr, P_pp = 0 and Q_qp = Q_pq^T for the
// orders that are not stored.  Left blocks B_1..B_k and right blocks C_{k+2}..C_{L-1}
// are updated (the ones the sweep uses before it rebuilds them).
void Engine::rotate_block_ops(int k, double theta) {
  const double c = std::cos(theta), s = std::sin(theta);
  // row x of U on spin-orbitals: (y, U_xy)
  auto urow = [&](int x) {
    std::vector<std::pair<int, double>> r;
    const int site = x >> 1, sg = x & 1;
    if (site == k) {
      r.push_back({x, c});
      r.push_back({2 * (k + 1) + sg, s});
    } else if (site == k + 1) {
      r.push_back({2 * k + sg, -s});
      r.push_back({x, c});
    } else {
      r.push_back({x, 1.0});
    }
    return r;
  };
  auto rotated = [&](int x) { return (x >> 1) == k || (x >> 1) == k + 1; };
  struct Src { OpKey key; int trans; double coef; };
  auto update = [&](Block& B, bool left) {
    if (!B.valid || B.ops.n_elem == 0) return;
    OpSet& os = B.ops;
    std::vector<std::pair<OpKey, std::vector<Src>>> work;
    for (auto& kv : os.ops) {
      const OpKey& key = kv.first;
      std::vector<Src> src;
      if (left) {
        if (key.type != OP_S || !rotated(key.i)) continue;
        for (auto& y : urow(key.i)) src.push_back(Src{OpKey{OP_S, y.first, 0}, 0, y.second});
      } else if (key.type == OP_T) {
        if (!rotated(key.i)) continue;
        for (auto& y : urow(key.i)) src.push_back(Src{OpKey{OP_T, y.first, 0}, 0, y.second});
      } else if (key.type == OP_P) {
        if (!rotated(key.i) && !rotated(key.j)) continue;
        for (auto& y1 : urow(key.i))
          for (auto& y2 : urow(key.j)) {
            if (y1.first == y2.first) continue;
            const double u = y1.second * y2.second;
            if (y1.first < y2.first) src.push_back(Src{OpKey{OP_P, y1.first, y2.first}, 0, u});
            else src.push_back(Src{OpKey{OP_P, y2.first, y1.first}, 0, -u});
          }
      } else if (key.type == OP_Q) {
        if (!rotated(key.i) && !rotated(key.j)) continue;
        for (auto& y1 : urow(key.i))
          for (auto& y2 : urow(key.j)) {
            const double u = y1.second * y2.second;
            if (y1.first <= y2.first) src.push_back(Src{OpKey{OP_Q, y1.first, y2.first}, 0, u});
            else src.push_back(Src{OpKey{OP_Q, y2.first, y1.first}, 1, u});
          }
      } else {
        continue;
      }
      work.push_back({key, src});
    }
    if (work.empty()) return;
    double* scratch = static_cast<double*>(ex_->alloc(size_t(os.n_elem) * sizeof(double)));
    std::vector<KronGroup> g;
    std::vector<KronTask> tk;
    for (auto& w : work) {
      const Op& tgt = os.ops.at(w.first);
      for (const OpBlk& tb : tgt.blk) {
        KronGroup kg;
        kg.dst = scratch + tb.off;
        kg.ld = tb.cols;
        kg.rows = tb.rows;
        kg.cols = tb.cols;
        kg.accumulate = 0;
        kg.t0 = int(tk.size());
        for (const Src& sr : w.second) {
          auto it = os.ops.find(sr.key);
          if (it == os.ops.end()) continue;
          const Op& so = it->second;
          // block (tb.r <- tb.c) of the source, or of its transpose
          const int want_c = sr.trans ? tb.r : tb.c, want_r = sr.trans ? tb.c : tb.r;
          auto bc = so.by_col.find(want_c);
          if (bc == so.by_col.end()) continue;
          const OpBlk& sb = so.blk[bc->second];
          if (sb.r != want_r) continue;
          tk.push_back(KronTask{os.arena + sb.off, sb.cols, sr.trans, sr.coef});
        }
        kg.t1 = int(tk.size());
        g.push_back(kg);
      }
    }
    if (!g.empty()) ex_->kron(g, tk);
    for (auto& w : work) {
      const Op& tgt = os.ops.at(w.first);
      for (const OpBlk& tb : tgt.blk)
        ex_->d2d(os.arena + tb.off, scratch + tb.off, size_t(tb.rows) * tb.cols * sizeof(double));
    }
    ex_->release(scratch);
  };
  for (int n = 1; n <= k; ++n) update(lb_[n], true);
  for (int m = k + 2; m < P_.L; ++m) update(rb_[m], false);
}

void Engine::set_state(const double* psi) {
  if (bond_ < 0) throw std::runtime_error("set_state: no bond prepared");
  if (!psi_cur_ || psi_cur_cap_ < psi_n_) {
    if (psi_cur_) ex_->release(psi_cur_);
    psi_cur_ = static_cast<double*>(ex_->alloc(size_t(psi_n_) * sizeof(double)));
  }
  psi_cur_cap_ = psi_n_;
  ex_->d2d(psi_cur_, psi, size_t(psi_n_) * sizeof(double));
  ex_->sync();
}

void Engine::apply_rotation(double theta) {
  if (bond_ < 0 || !psi_cur_) throw std::runtime_error("apply_rotation: no swept state");
  if (theta == 0.0) return;
  const int b = bond_;
  double* tmp = static_cast<double*>(ex_->alloc(size_t(psi_n_) * sizeof(double)));
  rotate_two_site(theta, psi_cur_, tmp);
  ex_->d2d(psi_cur_, tmp, size_t(psi_n_) * sizeof(double));
  ex_->release(tmp);
  // new integrals, the stored block operators rotated in place, the enlarged
  // operators and plans of the bond rebuilt
  rotate_integrals_pair(b, theta, false);
  rotate_block_ops(b, theta);
  prepare_bond(b);
}

double Engine::mode_step(double* s_before, double* s_after) {
  if (bond_ < 0 || !psi_cur_) throw std::runtime_error("mode_step: no swept state");
  double smin = 0.0, s0 = 0.0;
  const double theta = best_rotation(psi_cur_, &smin, &s0);
  apply_rotation(theta);
  if (s_before) *s_before = s0;
  if (s_after) *s_after = smin;
  return theta;
}

}  // namespace dmrg
