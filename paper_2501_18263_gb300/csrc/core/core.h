// Host core of the two-site U(1)xU(1) DMRG sigma engine (Sec. 2.3, Eqs.
// Hamilton_act_nonsym / Hamilton_act_U1sym): sector tables, the catalogue of
// normal and complementary block operators, the blocking / renormalisation /
// sigma / wave-function-transformation plans, and the Davidson and sweep
// drivers.  Everything numerical is delegated to an Exec (exec.h).
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../exec.h"

namespace dmrg {

// Runs f(i) for every i in [0, n) on up to 16 host threads, indices handed out
// one at a time (the calls must be independent: each writes only its own
// results).  The first exception is rethrown on the calling thread.
template <class F>
void host_parallel_for(int n, F&& f) {
  int nt = int(std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 16u));
  nt = std::min(nt, n);
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int> next{0};
  std::exception_ptr err;
  std::mutex mu;
  auto work = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) return;
      try {
        f(i);
      } catch (...) {
        std::lock_guard<std::mutex> g(mu);
        if (!err) err = std::current_exception();
        next.store(n);
        return;
      }
    }
  };
  std::vector<std::thread> th;
  th.reserve(size_t(nt - 1));
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  if (err) std::rethrow_exception(err);
}

struct QN {
  int a = 0, b = 0;  // n_alpha, n_beta
  bool operator<(const QN& o) const { return a < o.a || (a == o.a && b < o.b); }
  bool operator==(const QN& o) const { return a == o.a && b == o.b; }
  bool operator!=(const QN& o) const { return !(*this == o); }
  QN operator+(const QN& o) const { return {a + o.a, b + o.b}; }
  QN operator-(const QN& o) const { return {a - o.a, b - o.b}; }
  int n() const { return a + b; }
};

// local states of one orbital: 0 empty, 1 beta, 2 alpha, 3 alpha beta (= a+_a a+_b |0>)
extern const QN kLocalQ[4];

struct Sectors {
  std::vector<QN> q;
  std::vector<int> dim;
  std::vector<int64_t> off;
  int64_t total = 0;
  void finalize();
  int find(const QN& x) const;  // -1 if absent
};

// Enlarged block: left (block (x) site) or right (site (x) block).  Coarse
// sectors Q hold fine sub-blocks for s = 0..3 ascending.
struct Enlarged {
  bool left = true;
  Sectors coarse;
  // fine sectors, ordered by (coarse, s)
  std::vector<int> f_coarse, f_s, f_part, f_dim, f_row;
  std::vector<std::vector<int>> coarse_fines;
  std::vector<std::vector<int>> part_s_to_fine;  // [part][s] -> fine or -1
  void build(const Sectors& part, bool is_left);
  QN fq(int f) const { return coarse.q[f_coarse[f]]; }
};

enum OpType { OP_H = 0, OP_C, OP_A, OP_B, OP_S, OP_T, OP_P, OP_Q };

struct OpKey {
  int type, i, j;
  bool operator<(const OpKey& o) const {
    if (type != o.type) return type < o.type;
    if (i != o.i) return i < o.i;
    return j < o.j;
  }
};

struct OpBlk {
  int r, c;          // row / col sector (block sectors, or fine sectors on enlarged blocks)
  int rows, cols;
  int64_t off;       // element offset in the owning arena
  int ident = 0;     // enlarged only: block is c * identity (never read as a matrix)
  int64_t pn = -1, pt = -1;  // split-BF16 plane offsets: normal and transposed copies
};

struct Op {
  QN delta;
  int odd = 0;
  std::vector<OpBlk> blk;
  std::map<int, int> by_col;   // col sector -> index in blk  (one block per column sector)
  std::map<int, int> by_row;
};

struct OpSet {
  std::map<OpKey, Op> ops;
  double* arena = nullptr;
  int64_t n_elem = 0;
  const Op* get(int type, int i, int j = 0) const {
    auto it = ops.find(OpKey{type, i, j});
    return it == ops.end() ? nullptr : &it->second;
  }
};

// A coefficient that is linear in the integrals, c0 + sum_k w_k x_{idx_k}, with
// idx = i L + j for t_ij and L^2 + ((i L + j) L + k) L + l for (ij|kl) (chain order).
struct Lin {
  double c0 = 0.0;
  std::vector<std::pair<int64_t, double>> w;
};

// 4x4 matrix on one orbital with definite fermion parity; entries are numbers
// (N = double) or linear forms in the integrals (N = Lin)
template <class N>
struct Site4T {
  N m[4][4] = {};
  int odd = 0;
  bool zero() const;
};
using Site4 = Site4T<double>;

// One contribution of the blocking step, recorded for the adjoint: fine block
// (rf, cf) of the enlarged operator `key` receives coef * (block src_blk of the
// block operator src, transposed if trans; src == nullptr: the identity on the
// block part) (x) a site-matrix entry, the entry and the Jordan-Wigner sign
// folded into coef.
struct BlockingTerm {
  OpKey key;
  int rf, cf;
  const Op* src;
  int src_blk, trans;
  Lin coef;
};

// One term of H_eff at a bond: c * op(L) (x) op(R), op = transpose if Lt / Rt,
// nullptr = the identity on that side (Eq. Hamilton_act_U1sym)
struct SigmaTerm {
  const Op* L;
  int Lt;
  const Op* R;
  int Rt;
  double c;
};

struct Problem {
  int L = 0, na = 0, nb = 0;
  std::vector<double> t, v;  // permuted into chain order
  std::vector<int> ord;      // chain position -> orbital of the caller's numbering
  int D = 0;
  uint64_t seed = 0;
  int precision = 0;
  size_t mem_cap = 0;
  double h(int p, int q) const;                 // spin-orbital one-body
  double g(int p, int q, int r, int s) const;   // spin-orbital (pq|rs)
};

struct Block {
  bool valid = false;
  Sectors sec;
  OpSet ops;
};

struct Iso {  // site isometry: enlarged coarse sector -> new block sector
  bool valid = false;
  Sectors out;                     // new block sectors
  std::vector<double*> mat;        // per out sector: rows(enlarged Q) x out.dim, row-major
  std::vector<int> rows;
  double* arena = nullptr;
};

struct BondStats {
  int64_t psi_size = 0;
  int n_terms = 0;
  int64_t flops_stage1 = 0, flops_stage2 = 0;
  int64_t op_bytes = 0;   // algorithmic operator bytes read by one sigma (FP64)
  int n_gemm_problems = 0, n_gemm_segments = 0;
  int launches_per_sigma = 0;
  // split-BF16 plan: tiles and K stages (32 wide) of stage 1 / stage 2, X elements, plane bytes
  int64_t mix_tiles1 = 0, mix_steps1 = 0, mix_tiles2 = 0, mix_steps2 = 0, mix_x_elems = 0, mix_plane_bytes = 0;
  // which code paths the plan uses: term chunks (FP64 / split-BF16), split-K parts
  // of stage 2, stage-1 problems with several contributing fine blocks (mode 2) and
  // gathered-row problems (mode 3), the largest coarse L' dimension of psi, and the
  // stage-2 problems with more than one 128-row tile
  int64_t n_chunks = 0, mix_chunks = 0, mix_parts = 0, mix_mode2 = 0, mix_mode3 = 0, max_rows = 0,
          mix_multirow = 0;
};

class Engine {
 public:
  Engine(const Problem& p, Exec* ex);
  ~Engine();

  const Problem& problem() const { return P_; }
  Exec* exec() { return ex_; }

  // MPS basis input: sector tables of B_0..B_bond / C_{bond+2}..C_L and the
  // isometries of sites 0..bond-1 / bond+2..L-1 (host arrays).
  void load_left(int site, const Sectors& out, const std::vector<const double*>& mats);
  void load_right(int site, const Sectors& out, const std::vector<const double*>& mats);
  // whether B_n / C_m exists or can be built from the isometries held (loaded or swept)
  bool left_buildable(int n) const;
  bool right_buildable(int m) const;
  void build_left_blocks(int upto);     // B_0 .. B_upto from the loaded left isometries
  void build_right_blocks(int downto);  // C_L .. C_downto

  // bond workspace
  void prepare_bond(int bond);
  int bond() const { return bond_; }
  const std::vector<int64_t>& layout() const { return lay_; }   // rows of 7 ints (see ABI)
  int64_t psi_size() const { return psi_n_; }
  const BondStats& stats() const { return st_; }

  void sigma(const double* psi, double* sig);                 // device pointers, FP64 path
  void sigma_body(int precision);   // kernels of one sigma, psi_in_ -> sig_out_
  // the same, from the bond's captured graph when possible (captured on first use
  // unless allow_capture is false: capturing instantiates a graph)
  void sigma_run(int precision, bool allow_capture = true);
  // sharded sigma: per-term work (sigma_terms() order, then the local term H_L' (x) 1)
  // and the FP64 sigma of the terms with own[nu] != 0
  std::vector<int64_t> term_work() const;
  void sigma_subset(const double* psi, double* sig, const std::vector<char>& own);
  void sigma_precision(const double* psi, double* sig, int precision, bool allow_capture = true);
  void diagonal(double* d);                                    // diag of H_eff (device)

  // Davidson on the current bond; psi in/out (device).  Returns energy.  Sets
  // last_status: 0 converged (residual <= tol; for the split-BF16 sigma with
  // refine = 1, after an FP64 refinement), 1 stopped at the residual floor of the
  // split-BF16 sigma (refine = 0 only), 2 max_iter reached, 3 no new direction
  // (the subspace is invariant).
  double davidson(double* psi, double tol, int max_iter, int max_sub, int* iters_out, int refine);

  // sweeps.  flags bit 0: FP64 refinement at every step of a split-BF16 sweep
  // (otherwise only at the step whose energy is reported); bit 1: mode
  // optimisation micro-step after the eigensolver at every left-to-right step;
  // bit 2: a layer of swap gates on each half sweep (even bonds when first
  // visited, odd bonds on the way back), diagonalisation omitted there
  void init_sweep_state();
  std::vector<double> run_sweeps(int n, const int* Dsched, double tol, int flags = 0, int max_iter = 100);

  // expose a block operator for tests
  const Block& left_block(int n) const { return lb_[n]; }
  const Block& right_block(int m) const { return rb_[m]; }

  // Derivatives of F = <lam| H_eff(t, v) |psi> at the prepared bond, for the
  // fixed MPS basis, with respect to the integrals as this engine reads them (chain
  // order): raw[i L + j] = dF/dt_ij, raw[L^2 + ((i L + j) L + k) L + l] =
  // dF/dv_ijkl (host vector of L^2 + L^4).  Reverse mode through the sigma terms,
  // the blocking steps and the renormalisations of both block chains.
  void integral_gradient(const double* lam, const double* psi, std::vector<double>& raw);
  // blocking contributions with their coefficients as linear forms (adjoint)
  std::vector<BlockingTerm> blocking_terms(bool left, const Block& blk, int site, Enlarged& E) const;
  double lin_value(const Lin& c) const;
  // replace the integrals (chain order) and drop every block operator built from
  // the old ones; the loaded / swept isometries are kept
  void set_integrals(const std::vector<double>& t, const std::vector<double>& v);
  // wave function of the last sweep (device, at bond(); nullptr before a sweep)
  const double* sweep_psi() const { return psi_cur_; }
  // make psi (device, psi_size of the prepared bond) the current state
  void set_state(const double* psi);

  // mode optimisation (Sec. 2.2, Fig. 1; modeopt.cpp): psi in the orbitals rotated
  // by theta at the two sites of the prepared bond; the half-Renyi entropy of the
  // cut between them; the angle that minimises it; the micro-step on the swept
  // state (rotate psi and the integrals, rebuild the operators); returns theta
  void rotate_two_site(double theta, const double* in, double* out);
  std::vector<double> left_spectrum(const double* psi);
  double half_renyi(const double* psi);
  double entropy_at(double theta, const double* psi, double* scratch);
  double best_rotation(const double* psi, double* s_min, double* s0);
  void rotate_integrals_pair(int k, double theta, bool rebuild);
  void rotate_block_ops(int k, double theta);
  double mode_step(double* s_before, double* s_after);
  void apply_rotation(double theta);   // rotate the swept state and the integrals at bond()
  const std::vector<double>& chain_t() const { return P_.t; }
  const std::vector<double>& chain_v() const { return P_.v; }
  struct ModeLog { int sweep, bond; double theta, s_before, s_after; };
  std::vector<ModeLog> mode_log_;

  double last_energy = 0.0;
  double last_rnorm = 0.0;
  int last_status = 0;
  struct StepLog {
    int sweep, bond, ltr;
    double energy;
    int iters, status;
    double rnorm, discarded;
    std::vector<int> kept;   // sectors of the new block: (n_alpha, n_beta, dim) triples
  };
  std::vector<StepLog> sweep_log_;
  // wall seconds of the last run_sweeps call per phase (Sec. 4.1 categories):
  // 0 Tables (sigma plans), 1 Diag_H (Davidson), 2 SVD (density matrices,
  // eigensolver, selection), 3 Ren (renormalisation and enlargement), 4 StVec
  double phase_s[5] = {0, 0, 0, 0, 0};
  void set_D(int D) { P_.D = D; }
  // phase clock: while a sweep is timed, tick(k) charges the advance of the
  // device timeline since the last tick to phase k (a stream timestamp, no
  // synchronisation: the host may run ahead and build the next plans while the
  // device works; the phases are summed from the timestamps when the sweep ends)
  void tick(int k);
  void set_precision(int p) { P_.precision = p; }
  int64_t graph_runs() const { return graph_runs_; }

  // Batched form: the split-BF16 sigma of the prepared bond as separate steps,
  // so that the tensor-core tiles of several problems can share one grouped
  // launch per stage.  Valid while batchable() (one term chunk); the plan ids
  // are the executor's, and plan_generation() changes whenever they are rebuilt.
  bool batchable() const { return bond_ >= 0 && mixed_ready_ && mchunks_.size() == 1; }
  int mix_plan_hl() const { return mplan_hl_; }
  int mix_plan1() const { return mchunks_.empty() ? -1 : mchunks_[0].plan1; }
  int mix_plan2() const { return mchunks_.empty() ? -1 : mchunks_[0].plan2; }
  uint64_t plan_generation() const { return plan_gen_; }
  void batch_prologue(const double* psi);   // psi (device) -> split operand planes
  void batch_zero_parts();                  // clear the split-K part slots
  void batch_epilogue(double* sig);         // parts -> FP64 sigma (device)

 private:
  bool timing_ = false;
  std::vector<std::pair<int, int>> phase_marks_;   // (phase, stamp) at every tick of a timed sweep
  uint64_t plan_gen_ = 0;
  Problem P_;
  Exec* ex_;
  std::vector<Block> lb_, rb_;
  std::vector<Iso> liso_, riso_;
  int bond_ = -1;
  int lb_sec_known_ = 0;
  Enlarged EL_, ER_;
  OpSet EopsL_, EopsR_;
  std::vector<int64_t> lay_;
  std::vector<int64_t> psi_off_;       // per coarse L' sector: offset of psi block or -1
  std::vector<int> psi_rcoarse_;       // per coarse L' sector: coarse R' sector or -1
  int64_t psi_n_ = 0;
  BondStats st_;
  // sigma plan
  struct Chunk { int plan1 = -1; int plan2 = -1; };
  std::vector<Chunk> chunks_;
  int plan_hl_ = -1;
  double* xbuf_ = nullptr;
  double* psi_in_ = nullptr;
  double* sig_out_ = nullptr;
  int diag_plan_ = -1;
  std::vector<DiagTask> diag_tasks_;
  double* diag_l_ = nullptr;
  double* diag_r_ = nullptr;
  double* diag_ = nullptr;
  // split-BF16 tensor-core sigma
  bool mixed_ready_ = false;
  // blocked split matrices (three BF16 planes each) and the element counts of
  // their arenas
  uint16_t* oplL_ = nullptr;    // H_L' on coarse blocks
  uint16_t* oplR_ = nullptr;    // R' operators on coarse blocks, normal and transposed
  uint16_t* oplLf_ = nullptr;   // L' operators per fine sub-block, normal and transposed
  int64_t opsL_ = 0, opsR_ = 0, opsLf_ = 0;
  uint16_t* psiT_ = nullptr;    // psi^T per fine row block of L'
  uint16_t* psiN_ = nullptr;    // psi and psi^T per coarse block (local terms)
  int64_t psT_n_ = 0, psN_n_ = 0;
  uint16_t* xpl_ = nullptr;     // stage-1 results X
  int64_t xpl_n_ = 0;
  float* shi_ = nullptr;
  float* slo_ = nullptr;
  int psi_split_ = -1;
  std::vector<Chunk> mchunks_;
  int mplan_hl_ = -1;
  float* part_ = nullptr;
  int nparts_ = 1;
  // one captured CUDA graph per prepared bond and precision for the sigma steps of
  // Davidson (psi copied into psi_in_, result read from sig_out_ around the replay)
  int graph_[2] = {-1, -1};
  int64_t graph_runs_ = 0;
  void free_mixed();
  // sweep state
  double* psi_cur_ = nullptr;
  int64_t psi_cur_cap_ = 0;

  void free_opset(OpSet& s);
  void alloc_opset(OpSet& s);
  void enlarge(bool left, const Block& blk, int site, Enlarged& E, OpSet& out);
  void renormalize(bool left, const Enlarged& E, const OpSet& eops, const Iso& iso, Block& out);
  void build_sigma_plan();
  std::vector<SigmaTerm> sigma_terms(bool keep_empty = false) const;   // terms of the prepared bond (all but H_L' (x) 1)
  void sigma_adjoint(const double* lam, const double* psi, const std::map<OpKey, std::map<std::pair<int, int>, int64_t>>& tl,
                     double* gl, const std::map<OpKey, std::map<std::pair<int, int>, int64_t>>& tr, double* gr);
  void free_bond();
  void truncate_and_move(bool left_to_right, int D, double* trunc_w, std::vector<int>* kept = nullptr);
};

// site matrices
Site4 site_cdag(int sigma);
Site4 site_mul(const Site4& x, const Site4& y);
Site4 site_T(const Site4& x);
Site4 site_axpy(const Site4& x, double c, const Site4& y);  // x + c y

}  // namespace dmrg
