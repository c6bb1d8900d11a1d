// Sector tables, the operator catalogue and the two blocking steps (block (x)
// site, site (x) block) that build the normal and complementary operators of
// an enlarged block (Sec. 2.3: operators O^(nu,i) per subsystem, U(1)xU(1)
// block-sparse storage O{p}).  Renormalisation with a site isometry follows.
//
// Conventions.  Spin-orbital p = 2*site + sigma (sigma 0 alpha, 1 beta); the
// Jordan-Wigner order is ascending p.  With (pq|rs) the spin-orbital chemist
// integral (zero unless sigma_p = sigma_q and sigma_r = sigma_s):
//   H   = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs (pq|rs) a+_p a+_r a_s a_q
// Normal operators on a left block: C_p = a+_p, A_pr = a+_p a+_r (p<r),
//   B_pq = a+_p a_q (p<=q).
// Complementary operators (sums over the block's own spin-orbitals r,s,..):
//   S_q   = sum (pq|rs) a+_p a+_r a_s                  (left blocks, q outside)
//   T_p   = sum h_pq a_q + sum (pq|rs) a+_r a_s a_q    (right blocks, p outside)
//   P_pr  = sum (pq|rs) a_s a_q                        (right blocks, p<r outside)
//   Q_pq  = sum ((pq|rs) - (ps|rq)) a+_r a_s           (right blocks, p<=q outside)
// The bipartition L'|R' of the Hamiltonian into these terms is derived in the
// sigma plan (sigma.cpp).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>

#include "core.h"

namespace dmrg {

const QN kLocalQ[4] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};

void Sectors::finalize() {
  off.assign(q.size(), 0);
  total = 0;
  for (size_t i = 0; i < q.size(); ++i) {
    off[i] = total;
    total += dim[i];
  }
}

int Sectors::find(const QN& x) const {
  auto it = std::lower_bound(q.begin(), q.end(), x);
  if (it == q.end() || !(*it == x)) return -1;
  return int(it - q.begin());
}

void Enlarged::build(const Sectors& part, bool is_left) {
  left = is_left;
  std::map<QN, std::vector<std::pair<int, int>>> m;
  for (size_t k = 0; k < part.q.size(); ++k)
    for (int s = 0; s < 4; ++s) m[part.q[k] + kLocalQ[s]].push_back({s, int(k)});
  coarse = Sectors();
  f_coarse.clear(); f_s.clear(); f_part.clear(); f_dim.clear(); f_row.clear();
  coarse_fines.clear();
  part_s_to_fine.assign(part.q.size(), std::vector<int>(4, -1));
  for (auto& kv : m) {
    auto v = kv.second;
    std::sort(v.begin(), v.end());
    int ci = int(coarse.q.size());
    coarse.q.push_back(kv.first);
    int rows = 0;
    std::vector<int> fl;
    for (auto& sk : v) {
      int f = int(f_coarse.size());
      f_coarse.push_back(ci);
      f_s.push_back(sk.first);
      f_part.push_back(sk.second);
      f_dim.push_back(part.dim[sk.second]);
      f_row.push_back(rows);
      rows += part.dim[sk.second];
      part_s_to_fine[sk.second][sk.first] = f;
      fl.push_back(f);
    }
    coarse.dim.push_back(rows);
    coarse_fines.push_back(fl);
  }
  coarse.finalize();
}

// ---------------------------------------------------------------------------
// spin-orbital integrals

double Problem::h(int p, int q) const {
  if ((p & 1) != (q & 1)) return 0.0;
  return t[size_t(p >> 1) * L + (q >> 1)];
}

double Problem::g(int p, int q, int r, int s) const {
  if ((p & 1) != (q & 1) || (r & 1) != (s & 1)) return 0.0;
  size_t i = p >> 1, j = q >> 1, k = r >> 1, l = s >> 1;
  return v[((i * L + j) * L + k) * L + l];
}

// ---------------------------------------------------------------------------
// coefficients: numbers (the forward blocking) or linear forms in the integrals
// (the same blocking recorded for the adjoint)

namespace {

inline bool nz(double x) { return x != 0.0; }
inline bool nz(const Lin& x) { return x.c0 != 0.0 || !x.w.empty(); }
inline Lin operator*(Lin a, double s) {
  a.c0 *= s;
  for (auto& p : a.w) p.second *= s;
  return a;
}
inline Lin operator*(double s, const Lin& a) { return a * s; }
inline Lin operator+(Lin a, const Lin& b) {
  a.c0 += b.c0;
  a.w.insert(a.w.end(), b.w.begin(), b.w.end());
  return a;
}
inline Lin operator-(const Lin& a, const Lin& b) { return a + b * -1.0; }
// every blocking coefficient is a constant times a linear form: never a product of two
inline Lin operator*(const Lin& a, const Lin& b) {
  if (a.w.empty()) return b * a.c0;
  if (b.w.empty()) return a * b.c0;
  throw std::runtime_error("blocking coefficient is not linear in the integrals");
}

// integral access in the coefficient type
template <class N>
struct Ints;
template <>
struct Ints<double> {
  const Problem& P;
  double h(int p, int q) const { return P.h(p, q); }
  double g(int p, int q, int r, int s) const { return P.g(p, q, r, s); }
};
template <>
struct Ints<Lin> {
  const Problem& P;
  Lin h(int p, int q) const {
    if ((p & 1) != (q & 1)) return Lin{};
    return Lin{0.0, {{int64_t(p >> 1) * P.L + (q >> 1), 1.0}}};
  }
  Lin g(int p, int q, int r, int s) const {
    if ((p & 1) != (q & 1) || (r & 1) != (s & 1)) return Lin{};
    const int64_t L = P.L, i = p >> 1, j = q >> 1, k = r >> 1, l = s >> 1;
    return Lin{0.0, {{L * L + ((i * L + j) * L + k) * L + l, 1.0}}};
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// one-orbital matrices (basis 0, beta, alpha, alpha beta)

template <class N>
bool Site4T<N>::zero() const {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (nz(m[i][j])) return false;
  return true;
}
template struct Site4T<double>;
template struct Site4T<Lin>;

Site4 site_cdag(int sigma) {
  Site4 x;
  x.odd = 1;
  if (sigma == 0) {          // a+_alpha: |0> -> |a>, |b> -> |ab>
    x.m[2][0] = 1.0;
    x.m[3][1] = 1.0;
  } else {                   // a+_beta: |0> -> |b>, |a> -> -|ab>
    x.m[1][0] = 1.0;
    x.m[3][2] = -1.0;
  }
  return x;
}

Site4 site_T(const Site4& a) {
  Site4 x;
  x.odd = a.odd;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) x.m[i][j] = a.m[j][i];
  return x;
}

Site4 site_mul(const Site4& a, const Site4& b) {
  Site4 x;
  x.odd = a.odd ^ b.odd;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0;
      for (int k = 0; k < 4; ++k) s += a.m[i][k] * b.m[k][j];
      x.m[i][j] = s;
    }
  return x;
}

Site4 site_axpy(const Site4& a, double c, const Site4& b) {
  Site4 x = a;
  if (a.zero()) x.odd = b.odd;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) x.m[i][j] += c * b.m[i][j];
  return x;
}

static Site4 site_id() {
  Site4 x;
  for (int i = 0; i < 4; ++i) x.m[i][i] = 1.0;
  return x;
}

namespace {

// x + c y for a constant matrix y (entries of y that are zero add nothing)
template <class N>
Site4T<N> axpy(const Site4T<N>& a, const N& c, const Site4& b) {
  Site4T<N> x = a;
  if (a.zero()) x.odd = b.odd;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (b.m[i][j] != 0.0) x.m[i][j] = x.m[i][j] + c * b.m[i][j];
  return x;
}
template <class N>
Site4T<N> transpose(const Site4T<N>& a) {
  Site4T<N> x;
  x.odd = a.odd;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) x.m[i][j] = a.m[j][i];
  return x;
}
template <class N>
Site4T<N> lift(const Site4& a);
template <>
Site4 lift<double>(const Site4& a) { return a; }
template <>
Site4T<Lin> lift<Lin>(const Site4& a) {
  Site4T<Lin> x;
  x.odd = a.odd;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (a.m[i][j] != 0.0) x.m[i][j] = Lin{a.m[i][j], {}};
  return x;
}

template <class N>
struct SiteOps {
  Ints<N> I;
  int site;
  int X[2];
  Site4 cd[2], c[2];
  SiteOps(const Problem& p, int s) : I{p}, site(s) {
    X[0] = 2 * s;
    X[1] = 2 * s + 1;
    for (int k = 0; k < 2; ++k) {
      cd[k] = site_cdag(k);
      c[k] = site_T(cd[k]);
    }
  }
  const Site4& CD(int x) const { return cd[x & 1]; }
  const Site4& CC(int x) const { return c[x & 1]; }
  Site4 prod(const Site4& a, const Site4& b) const { return site_mul(a, b); }
  Site4 prod(const Site4& a, const Site4& b, const Site4& d) const { return site_mul(site_mul(a, b), d); }
  // H restricted to the orbital
  Site4T<N> H() const {
    Site4T<N> r;
    for (int p : X)
      for (int q : X) {
        const N h = I.h(p, q);
        if (nz(h)) r = axpy(r, h, prod(CD(p), CC(q)));
      }
    for (int p : X)
      for (int q : X)
        for (int rr : X)
          for (int s : X) {
            const N g = I.g(p, q, rr, s);
            if (nz(g)) r = axpy(r, g * 0.5, site_mul(prod(CD(p), CD(rr), CC(s)), CC(q)));
          }
    return r;
  }
  // T_p restricted to the orbital (p outside): sum_q h_pq a_q + sum_qrs (pq|rs) a+_r a_s a_q
  Site4T<N> T(int p) const {
    Site4T<N> r;
    r.odd = 1;
    for (int q : X) {
      const N h = I.h(p, q);
      if (nz(h)) r = axpy(r, h, CC(q));
    }
    for (int q : X)
      for (int rr : X)
        for (int s : X) {
          const N g = I.g(p, q, rr, s);
          if (nz(g)) r = axpy(r, g, prod(CD(rr), CC(s), CC(q)));
        }
    return r;
  }
  // S_q restricted to the orbital (q outside): sum_prs (pq|rs) a+_p a+_r a_s
  Site4T<N> S(int q) const {
    Site4T<N> r;
    r.odd = 1;
    for (int p : X)
      for (int rr : X)
        for (int s : X) {
          const N g = I.g(p, q, rr, s);
          if (nz(g)) r = axpy(r, g, prod(CD(p), CD(rr), CC(s)));
        }
    return r;
  }
  // P_pr restricted: sum_qs (pq|rs) a_s a_q
  Site4T<N> Pc(int p, int rr) const {
    Site4T<N> r;
    for (int q : X)
      for (int s : X) {
        const N g = I.g(p, q, rr, s);
        if (nz(g)) r = axpy(r, g, prod(CC(s), CC(q)));
      }
    return r;
  }
  // Q_pq restricted: sum_rs ((pq|rs) - (ps|rq)) a+_r a_s
  Site4T<N> Qc(int p, int q) const {
    Site4T<N> r;
    for (int rr : X)
      for (int s : X) {
        const N g = I.g(p, q, rr, s) - I.g(p, s, rr, q);
        if (nz(g)) r = axpy(r, g, prod(CD(rr), CC(s)));
      }
    return r;
  }
};

QN espin(int p) { return (p & 1) ? QN{0, 1} : QN{1, 0}; }

void key_qn(const OpKey& k, QN& d, int& odd) {
  switch (k.type) {
    case OP_H: d = {0, 0}; odd = 0; break;
    case OP_C: d = espin(k.i); odd = 1; break;
    case OP_A: d = espin(k.i) + espin(k.j); odd = 0; break;
    case OP_B: d = espin(k.i) - espin(k.j); odd = 0; break;
    case OP_S: d = espin(k.i); odd = 1; break;
    case OP_T: d = QN{0, 0} - espin(k.i); odd = 1; break;
    case OP_P: d = QN{0, 0} - espin(k.i) - espin(k.j); odd = 0; break;
    case OP_Q: d = espin(k.j) - espin(k.i); odd = 0; break;
  }
}

}  // namespace

std::vector<OpKey> left_keys(int n, int L) {
  std::vector<OpKey> k;
  k.push_back({OP_H, 0, 0});
  for (int p = 0; p < 2 * n; ++p) k.push_back({OP_C, p, 0});
  for (int p = 0; p < 2 * n; ++p)
    for (int r = p + 1; r < 2 * n; ++r) k.push_back({OP_A, p, r});
  for (int p = 0; p < 2 * n; ++p)
    for (int q = p; q < 2 * n; ++q) k.push_back({OP_B, p, q});
  for (int q = 2 * n; q < 2 * L; ++q) k.push_back({OP_S, q, 0});
  return k;
}

std::vector<OpKey> right_keys(int m, int L) {
  std::vector<OpKey> k;
  k.push_back({OP_H, 0, 0});
  for (int q = 2 * m; q < 2 * L; ++q) k.push_back({OP_C, q, 0});
  for (int p = 0; p < 2 * m; ++p) k.push_back({OP_T, p, 0});
  for (int p = 0; p < 2 * m; ++p)
    for (int r = p + 1; r < 2 * m; ++r) k.push_back({OP_P, p, r});
  for (int p = 0; p < 2 * m; ++p)
    for (int q = p; q < 2 * m; ++q) k.push_back({OP_Q, p, q});
  return k;
}

// Empty operator on a renormalised block with every block its quantum numbers allow.
static Op make_block_op(const Sectors& sec, const OpKey& key) {
  Op o;
  key_qn(key, o.delta, o.odd);
  for (size_t c = 0; c < sec.q.size(); ++c) {
    int r = sec.find(sec.q[c] + o.delta);
    if (r < 0) continue;
    OpBlk b;
    b.r = r;
    b.c = int(c);
    b.rows = sec.dim[r];
    b.cols = sec.dim[c];
    b.off = 0;
    o.by_col[b.c] = int(o.blk.size());
    o.by_row[b.r] = int(o.blk.size());
    o.blk.push_back(b);
  }
  return o;
}

void Engine::free_opset(OpSet& s) {
  if (s.arena) ex_->release(s.arena);
  s.arena = nullptr;
  s.n_elem = 0;
  s.ops.clear();
}

void Engine::alloc_opset(OpSet& s) {
  int64_t n = 0;
  for (auto& kv : s.ops)
    for (auto& b : kv.second.blk) {
      b.off = n;
      n += int64_t(b.rows) * b.cols;
    }
  s.n_elem = n;
  s.arena = n ? static_cast<double*>(ex_->alloc(size_t(n) * sizeof(double))) : nullptr;
}

// ---------------------------------------------------------------------------
// blocking: enlarged operator = sum of (block op) (x) (site matrix)

namespace {

template <class N>
struct Pend {
  const Op* src;      // nullptr: identity on the block
  const OpSet* set;
  int blk;            // block index in src (-1 for identity)
  int trans;
  N coef;
};

template <class N>
struct EnlOpBuild {
  Op op;
  std::map<std::pair<int, int>, std::vector<Pend<N>>> tgt;
};

template <class N>
struct Blocker {
  const Enlarged& E;
  const Sectors& part;
  const OpSet& src;
  bool left;
  Blocker(const Enlarged& e, const Sectors& p, const OpSet& s) : E(e), part(p), src(s), left(e.left) {}

  // target += coef * (op or identity, maybe transposed) (x) M   [left: block (x) site]
  //        += coef * M (x) (op ...)                              [right: site (x) block]
  void add(EnlOpBuild<N>& t, const Op* op, int trans, const Site4T<N>& M, const N& coef) {
    if (!nz(coef) || M.zero()) return;
    if (op && op->blk.empty()) return;
    int src_odd = op ? op->odd : 0;
    for (int s2 = 0; s2 < 4; ++s2)
      for (int s = 0; s < 4; ++s) {
        const N& mv = M.m[s2][s];
        if (!nz(mv)) continue;
        int nsite = kLocalQ[s].n();
        if (!op) {
          for (size_t k = 0; k < part.q.size(); ++k) {
            int rf = E.part_s_to_fine[k][s2], cf = E.part_s_to_fine[k][s];
            double sg = 1.0;
            if (left && M.odd && (part.q[k].n() & 1)) sg = -1.0;
            t.tgt[{rf, cf}].push_back(Pend<N>{nullptr, &src, -1, 0, coef * mv * sg});
          }
        } else {
          for (size_t bi = 0; bi < op->blk.size(); ++bi) {
            const OpBlk& b = op->blk[bi];
            int rp = trans ? b.c : b.r, cp = trans ? b.r : b.c;
            int rf = E.part_s_to_fine[rp][s2], cf = E.part_s_to_fine[cp][s];
            double sg = 1.0;
            if (left) {
              if (M.odd && (part.q[cp].n() & 1)) sg = -1.0;
            } else {
              if (src_odd && (nsite & 1)) sg = -1.0;
            }
            t.tgt[{rf, cf}].push_back(Pend<N>{op, &src, int(bi), trans, coef * mv * sg});
          }
        }
      }
  }
};

template <class N>
N num(double x);
template <>
double num<double>(double x) { return x; }
template <>
Lin num<Lin>(double x) { return Lin{x, {}}; }

// The blocking step (block (x) site for a left block, site (x) block for a right
// one): every fine block of every operator of the enlarged block as a list of
// contributions coef * (block operator block, or the identity) (x) site matrix
// entry.  N = double gives the numbers; N = Lin the same list with every
// coefficient kept as a linear form in the integrals.
template <class N>
std::map<OpKey, EnlOpBuild<N>> collect_blocking(const Problem& P, bool left, const Block& blk, int site,
                                                Enlarged& E) {
  E.build(blk.sec, left);
  const int L = P.L;
  SiteOps<N> so(P, site);
  const Ints<N>& I = so.I;
  const int X0 = 2 * site, X1 = 2 * site + 1;
  const int X[2] = {X0, X1};
  const Site4 I4 = site_id();
  const N one = num<N>(1.0), mone = num<N>(-1.0);
  Blocker<N> bl(E, blk.sec, blk.ops);
  static const Op kEmpty;  // absent operator = zero (never the identity)
  auto G = [&](int t, int i, int j = 0) -> const Op* {
    const Op* o = blk.ops.get(t, i, j);
    return o ? o : &kEmpty;
  };
  // B_ps for any order (transposed storage for p > s)
  auto addB = [&](EnlOpBuild<N>& t, int p, int s, const Site4T<N>& M, const N& c) {
    if (p <= s) bl.add(t, G(OP_B, p, s), 0, M, c);
    else bl.add(t, G(OP_B, s, p), 1, M, c);
  };

  std::map<OpKey, EnlOpBuild<N>> build;
  std::vector<OpKey> keys = left ? left_keys(site + 1, L) : right_keys(site, L);
  std::vector<EnlOpBuild<N>*> tp(keys.size());
  for (size_t i = 0; i < keys.size(); ++i) {
    tp[i] = &build[keys[i]];
    key_qn(keys[i], tp[i]->op.delta, tp[i]->op.odd);
  }
  // every operator's contributions are collected on their own (host threads; the
  // block, the site operators and the integrals are only read)

  if (left) {
    const int nB = 2 * site;  // block spin-orbitals [0, nB)
    host_parallel_for(int(keys.size()), [&](int ki) {
      const OpKey& k = keys[ki];
      EnlOpBuild<N>& t = *tp[ki];
      switch (k.type) {
        case OP_H: {
          bl.add(t, G(OP_H, 0), 0, lift<N>(I4), one);
          bl.add(t, nullptr, 0, so.H(), one);
          for (int p = 0; p < nB; ++p) {
            Site4T<N> Tp = so.T(p);
            bl.add(t, G(OP_C, p), 0, Tp, one);
            bl.add(t, G(OP_C, p), 1, transpose(Tp), mone);
          }
          for (int q : X) {
            bl.add(t, G(OP_S, q), 0, lift<N>(so.CC(q)), one);
            bl.add(t, G(OP_S, q), 1, lift<N>(so.CD(q)), mone);
          }
          for (int p = 0; p < nB; ++p)
            for (int r = p + 1; r < nB; ++r) {
              Site4T<N> Pm = so.Pc(p, r);
              bl.add(t, G(OP_A, p, r), 0, Pm, one);
              bl.add(t, G(OP_A, p, r), 1, transpose(Pm), one);
            }
          for (int p = 0; p < nB; ++p)
            for (int q = p; q < nB; ++q) {
              Site4T<N> Qm = so.Qc(p, q);
              bl.add(t, G(OP_B, p, q), 0, Qm, one);
              if (p < q) bl.add(t, G(OP_B, p, q), 1, transpose(Qm), one);
            }
          break;
        }
        case OP_C:
          if (k.i < nB) bl.add(t, G(OP_C, k.i), 0, lift<N>(I4), one);
          else bl.add(t, nullptr, 0, lift<N>(so.CD(k.i)), one);
          break;
        case OP_A:
          if (k.j < nB) bl.add(t, G(OP_A, k.i, k.j), 0, lift<N>(I4), one);
          else if (k.i < nB) bl.add(t, G(OP_C, k.i), 0, lift<N>(so.CD(k.j)), one);
          else bl.add(t, nullptr, 0, lift<N>(so.prod(so.CD(k.i), so.CD(k.j))), one);
          break;
        case OP_B:
          if (k.j < nB) bl.add(t, G(OP_B, k.i, k.j), 0, lift<N>(I4), one);
          else if (k.i < nB) bl.add(t, G(OP_C, k.i), 0, lift<N>(so.CC(k.j)), one);
          else bl.add(t, nullptr, 0, lift<N>(so.prod(so.CD(k.i), so.CC(k.j))), one);
          break;
        case OP_S: {
          const int q = k.i;
          bl.add(t, G(OP_S, q), 0, lift<N>(I4), one);
          bl.add(t, nullptr, 0, so.S(q), one);
          // two block operators, one site operator
          for (int s : X)
            for (int p = 0; p < nB; ++p)
              for (int r = p + 1; r < nB; ++r) {
                const N c = I.g(p, q, r, s) - I.g(r, q, p, s);
                if (nz(c)) bl.add(t, G(OP_A, p, r), 0, lift<N>(so.CC(s)), c);
              }
          for (int x : X)
            for (int p = 0; p < nB; ++p)
              for (int s = 0; s < nB; ++s) {
                const N c = I.g(x, q, p, s) - I.g(p, q, x, s);
                if (nz(c)) addB(t, p, s, lift<N>(so.CD(x)), c);
              }
          // one block operator, two site operators
          for (int y = 0; y < nB; ++y) {
            Site4T<N> M1, M2;
            for (int r : X)
              for (int s : X) {
                const N c = I.g(y, q, r, s) - I.g(r, q, y, s);
                if (nz(c)) M1 = axpy(M1, c, so.prod(so.CD(r), so.CC(s)));
              }
            for (int p : X)
              for (int r : X) {
                const N c = I.g(p, q, r, y);
                if (nz(c)) M2 = axpy(M2, c, so.prod(so.CD(p), so.CD(r)));
              }
            bl.add(t, G(OP_C, y), 0, M1, one);
            bl.add(t, G(OP_C, y), 1, M2, one);
          }
          break;
        }
        default:
          throw std::runtime_error("left enlargement: unexpected operator");
      }
    });
  } else {
    const int c0 = 2 * (site + 1);  // block spin-orbitals [c0, 2L)
    host_parallel_for(int(keys.size()), [&](int ki) {
      const OpKey& k = keys[ki];
      EnlOpBuild<N>& t = *tp[ki];
      switch (k.type) {
        case OP_H: {
          bl.add(t, G(OP_H, 0), 0, lift<N>(I4), one);
          bl.add(t, nullptr, 0, so.H(), one);
          for (int p : X) {
            bl.add(t, G(OP_T, p), 0, lift<N>(so.CD(p)), one);
            bl.add(t, G(OP_T, p), 1, lift<N>(so.CC(p)), mone);
          }
          for (int q = c0; q < 2 * L; ++q) {
            Site4T<N> Sq = so.S(q);
            bl.add(t, G(OP_C, q), 1, Sq, one);
            bl.add(t, G(OP_C, q), 0, transpose(Sq), mone);
          }
          {
            Site4 A = so.prod(so.CD(X0), so.CD(X1));
            bl.add(t, G(OP_P, X0, X1), 0, lift<N>(A), one);
            bl.add(t, G(OP_P, X0, X1), 1, lift<N>(site_T(A)), one);
          }
          for (int p : X)
            for (int q : X) {
              if (q < p) continue;
              Site4 Bm = so.prod(so.CD(p), so.CC(q));
              bl.add(t, G(OP_Q, p, q), 0, lift<N>(Bm), one);
              if (p < q) bl.add(t, G(OP_Q, p, q), 1, lift<N>(site_T(Bm)), one);
            }
          break;
        }
        case OP_C:
          if (k.i >= c0) bl.add(t, G(OP_C, k.i), 0, lift<N>(I4), one);
          else bl.add(t, nullptr, 0, lift<N>(so.CD(k.i)), one);
          break;
        case OP_T: {
          const int p = k.i;
          bl.add(t, nullptr, 0, so.T(p), one);
          bl.add(t, G(OP_T, p), 0, lift<N>(I4), one);
          for (int x : X) {
            bl.add(t, G(OP_Q, p, x), 0, lift<N>(so.CC(x)), one);
            bl.add(t, G(OP_P, p, x), 0, lift<N>(so.CD(x)), one);
          }
          for (int y = c0; y < 2 * L; ++y) {
            Site4T<N> M1, M2;
            for (int r : X)
              for (int s : X) {
                const N c = I.g(p, y, r, s) - I.g(p, s, r, y);
                if (nz(c)) M1 = axpy(M1, c, so.prod(so.CD(r), so.CC(s)));
              }
            for (int q : X)
              for (int s : X) {
                const N c = I.g(p, q, y, s);
                if (nz(c)) M2 = axpy(M2, c, so.prod(so.CC(s), so.CC(q)));
              }
            bl.add(t, G(OP_C, y), 1, M1, one);
            bl.add(t, G(OP_C, y), 0, M2, one);
          }
          break;
        }
        case OP_P: {
          const int p = k.i, r = k.j;
          bl.add(t, nullptr, 0, so.Pc(p, r), one);
          bl.add(t, G(OP_P, p, r), 0, lift<N>(I4), one);
          for (int x : X)
            for (int y = c0; y < 2 * L; ++y) {
              const N c = I.g(p, y, r, x) - I.g(p, x, r, y);
              if (nz(c)) bl.add(t, G(OP_C, y), 1, lift<N>(so.CC(x)), c);
            }
          break;
        }
        case OP_Q: {
          const int p = k.i, q = k.j;
          bl.add(t, nullptr, 0, so.Qc(p, q), one);
          bl.add(t, G(OP_Q, p, q), 0, lift<N>(I4), one);
          for (int x : X)
            for (int y = c0; y < 2 * L; ++y) {
              const N c1 = I.g(p, q, x, y) - I.g(p, y, x, q);
              if (nz(c1)) bl.add(t, G(OP_C, y), 1, lift<N>(so.CD(x)), c1);
              const N c2 = I.g(p, q, y, x) - I.g(p, x, y, q);
              if (nz(c2)) bl.add(t, G(OP_C, y), 0, lift<N>(so.CC(x)), c2 * -1.0);
            }
          break;
        }
        default:
          throw std::runtime_error("right enlargement: unexpected operator");
      }
    });
  }

  return build;
}

}  // namespace

std::vector<BlockingTerm> Engine::blocking_terms(bool left, const Block& blk, int site, Enlarged& E) const {
  std::map<OpKey, EnlOpBuild<Lin>> build = collect_blocking<Lin>(P_, left, blk, site, E);
  std::vector<BlockingTerm> out;
  for (auto& kv : build)
    for (auto& tg : kv.second.tgt)
      for (auto& pd : tg.second) {
        BlockingTerm bt{kv.first, tg.first.first, tg.first.second, pd.src, pd.blk, pd.trans, Lin{pd.coef.c0, {}}};
        // merge repeated integrals, drop zero weights
        std::map<int64_t, double> w;
        for (auto& x : pd.coef.w) w[x.first] += x.second;
        for (auto& x : w)
          if (x.second != 0.0) bt.coef.w.push_back(x);
        out.push_back(std::move(bt));
      }
  return out;
}

double Engine::lin_value(const Lin& c) const {
  const int64_t L2 = int64_t(P_.L) * P_.L;
  double x = c.c0;
  for (auto& w : c.w) x += w.second * (w.first < L2 ? P_.t[size_t(w.first)] : P_.v[size_t(w.first - L2)]);
  return x;
}

void Engine::enlarge(bool left, const Block& blk, int site, Enlarged& E, OpSet& out) {
  std::map<OpKey, EnlOpBuild<double>> build = collect_blocking<double>(P_, left, blk, site, E);

  // allocate the fine blocks that received contributions, then emit the kron plan
  free_opset(out);
  for (auto& kv : build) {
    EnlOpBuild<double>& t = kv.second;
    Op& o = t.op;
    for (auto& tg : t.tgt) {
      OpBlk b;
      b.r = tg.first.first;
      b.c = tg.first.second;
      b.rows = E.f_dim[b.r];
      b.cols = E.f_dim[b.c];
      b.ident = 1;
      for (auto& pd : tg.second)
        if (pd.src) b.ident = 0;
      o.blk.push_back(b);
    }
    out.ops[kv.first] = o;
  }
  alloc_opset(out);
  // one group per fine block, one task per contribution: every operator's first
  // group and task from prefix sums, then the lists filled on host threads
  std::vector<std::pair<const EnlOpBuild<double>*, Op*>> opl;
  std::vector<int64_t> goff(1, 0), toff(1, 0);
  for (auto& kv : build) {
    opl.push_back({&kv.second, &out.ops[kv.first]});
    int64_t nt = 0;
    for (auto& tg : kv.second.tgt) nt += int64_t(tg.second.size());
    goff.push_back(goff.back() + int64_t(kv.second.tgt.size()));
    toff.push_back(toff.back() + nt);
  }
  if (toff.back() > int64_t(INT32_MAX)) throw std::runtime_error("enlarge: too many blocking contributions");
  std::vector<KronGroup> groups(size_t(goff.back()));
  std::vector<KronTask> tasks(size_t(toff.back()));
  host_parallel_for(int(opl.size()), [&](int i) {
    Op& o = *opl[size_t(i)].second;
    size_t gi = size_t(goff[size_t(i)]), ti = size_t(toff[size_t(i)]);
    size_t bi = 0;
    for (auto& tg : opl[size_t(i)].first->tgt) {
      OpBlk& b = o.blk[bi++];
      o.by_col[b.c] = int(bi - 1);
      KronGroup g;
      g.dst = out.arena + b.off;
      g.ld = b.cols;
      g.rows = b.rows;
      g.cols = b.cols;
      g.t0 = int(ti);
      g.accumulate = 0;
      for (auto& pd : tg.second) {
        KronTask tk;
        if (!pd.src) {
          tk.src = nullptr;
          tk.src_ld = 0;
          tk.mode = 2;
        } else {
          const OpBlk& sb = pd.src->blk[pd.blk];
          tk.src = pd.set->arena + sb.off;
          tk.src_ld = sb.cols;
          tk.mode = pd.trans ? 1 : 0;
        }
        tk.coef = pd.coef;
        tasks[ti++] = tk;
      }
      g.t1 = int(ti);
      groups[gi++] = g;
    }
  });
  if (!groups.empty()) ex_->kron(groups, tasks);
}

// ---------------------------------------------------------------------------
// renormalisation: new = U^T O U, fine-block by fine-block

void Engine::renormalize(bool left, const Enlarged& E, const OpSet& eops, const Iso& iso, Block& out) {
  (void)left;
  free_opset(out.ops);
  out.sec = iso.out;
  out.valid = true;
  const Sectors& S = iso.out;
  std::vector<int> s2c(S.q.size());
  for (size_t k = 0; k < S.q.size(); ++k) {
    s2c[k] = E.coarse.find(S.q[k]);
    if (s2c[k] < 0 || E.coarse.dim[s2c[k]] != iso.rows[k])
      throw std::runtime_error("renormalize: isometry does not match the enlarged basis");
  }
  for (auto& kv : eops.ops) {
    Op o = make_block_op(S, kv.first);
    out.ops.ops[kv.first] = o;
  }
  alloc_opset(out.ops);

  // scratch for T1 = O U, processed in batches
  const int64_t cap = int64_t(1) << 27;  // elements (1 GiB)
  double* scratch = nullptr;
  int64_t scratch_n = 0;
  std::vector<GemmProb> p1, p2;
  std::vector<GemmSeg> s1, s2;
  int64_t used = 0;
  auto flush = [&]() {
    if (!p1.empty()) ex_->gemm(p1, s1);
    if (!p2.empty()) ex_->gemm(p2, s2);
    p1.clear(); p2.clear(); s1.clear(); s2.clear();
    used = 0;
  };
  for (auto& kv : eops.ops) {
    const Op& eo = kv.second;
    Op& no = out.ops.ops[kv.first];
    // index enlarged fine blocks by (row fine, col fine)
    std::map<std::pair<int, int>, const OpBlk*> fb;
    for (auto& b : eo.blk) fb[{b.r, b.c}] = &b;
    // estimate scratch need for this op
    int64_t need = 0;
    for (auto& nb : no.blk) need += int64_t(E.coarse.dim[s2c[nb.r]]) * S.dim[nb.c];
    if (used + need > scratch_n) {
      flush();
      if (need > scratch_n) {
        if (scratch) ex_->release(scratch);
        scratch_n = std::max(need, std::min(cap, int64_t(1) << 22));
        scratch = static_cast<double*>(ex_->alloc(size_t(scratch_n) * sizeof(double)));
      }
    }
    for (auto& nb : no.blk) {
      const int cr = s2c[nb.r], cc = s2c[nb.c];
      const double* Ur = iso.mat[nb.r];
      const double* Uc = iso.mat[nb.c];
      const int dr = S.dim[nb.r], dc = S.dim[nb.c];
      GemmProb q2;
      q2.C = out.ops.arena + nb.off;
      q2.ldc = dc;
      q2.M = dr;
      q2.N = dc;
      q2.alpha = 1.0;
      q2.accumulate = 0;
      q2.s0 = int(s2.size());
      for (int fr : E.coarse_fines[cr]) {
        GemmProb q1;
        q1.C = scratch + used;
        q1.ldc = dc;
        q1.M = E.f_dim[fr];
        q1.N = dc;
        q1.alpha = 1.0;
        q1.accumulate = 0;
        q1.s0 = int(s1.size());
        for (int fc : E.coarse_fines[cc]) {
          auto it = fb.find({fr, fc});
          if (it == fb.end()) continue;
          const OpBlk* b = it->second;
          s1.push_back(GemmSeg{eops.arena + b->off, Uc + int64_t(E.f_row[fc]) * dc, b->cols, dc,
                               b->cols, 0, 0});
        }
        q1.s1 = int(s1.size());
        if (q1.s1 == q1.s0) continue;
        p1.push_back(q1);
        s2.push_back(GemmSeg{Ur + int64_t(E.f_row[fr]) * dr, q1.C, dr, dc, E.f_dim[fr], 1, 0});
        used += int64_t(E.f_dim[fr]) * dc;
      }
      q2.s1 = int(s2.size());
      p2.push_back(q2);
    }
  }
  flush();
  if (scratch) ex_->release(scratch);
}

}  // namespace dmrg
