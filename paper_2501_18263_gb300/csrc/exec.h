// Numerical primitives the DMRG host core drives.  The product library
// implements them with sm_103a kernels (exec_cuda.cu); every pointer handed to
// them is a device pointer owned by the engine's arenas.
#pragma once
#include <cstddef>
#include <cstdint>
#include <functional>
#include <vector>

namespace dmrg {

// dst[r, c] (+)= sum_t coef_t * src_t[r, c]   (mode 0: src row-major, 1: src^T, 2: identity)
struct KronTask {
  const double* src;
  int src_ld;
  int mode;
  double coef;
};
struct KronGroup {
  double* dst;
  int ld, rows, cols;
  int t0, t1;        // task range in the task array
  int accumulate;    // 0: dst = sum, 1: dst += sum
};

// C = alpha * sum_seg op(A_seg) op(B_seg)  (+ C if accumulate)
// op(A) is M x K: ta = 0 -> A[m*lda + k], ta = 1 -> A[k*lda + m]
// op(B) is K x N: tb = 0 -> B[k*ldb + n], tb = 1 -> B[n*ldb + k]
struct GemmSeg {
  const double* A;
  const double* B;
  int lda, ldb, K, ta, tb;
};
struct GemmProb {
  double* C;
  int ldc, M, N;
  int s0, s1;        // segment range
  double alpha;
  int accumulate;
};

// element-wise diagonal extraction: dst[i * dst_stride] = coef * (src ? src[i*(ld+1)] : 1)
struct DiagTask {
  const double* src;
  int ld, n;
  double* dst;
  int64_t dst_stride;
  double coef;
};

// Frobenius products for the adjoint: out = sum_{r < rows, c < cols} a[r*lda + c] *
// (mode 0: b[r*ldb + c], mode 1: b[c*ldb + r], mode 2: 1 if r == c else 0)
struct DotTask {
  const double* a;
  const double* b;
  int lda, ldb, rows, cols, mode;
};

// ---- split-BF16 tensor-core path -------------------------------------------
// An operand x is carried as three BF16 planes (x ~ hi + mid + lo) stored
// together in a "blocked split matrix": for a matrix with R rows (R8 = R padded
// to 8) and K extent Kt (a multiple of 32), rows form blocks of 128 (the last
// one h = min(128, R8 - 128 rb) rows), each block is cut into K slabs of 32, and
// one slab holds, per 8-row group, the three planes' 8 x 32 pieces as 8 x 8 core
// matrices (8 rows x 16 bytes).  Element (plane q, row r, k) is at
//     rb * 384 Kt + (k / 32) * 96 h + (rr / 8) * 768 + q * 256
//       + ((k % 32) / 8) * 64 + (rr % 8) * 8 + k % 8,      rb = r / 128, rr = r % 128
// so the piece of a 128-row tile that one 32-wide K step needs (all three planes)
// is one contiguous run of 192 h bytes.  Padding rows and columns are zero.
#if defined(__CUDACC__)
#define DMRG_HD __host__ __device__
#else
#define DMRG_HD
#endif
DMRG_HD inline int64_t blk_off(int q, int r, int k, int R8, int Kt) {
  const int rb = r >> 7, rr = r & 127;
  const int h = (R8 - (rb << 7)) < 128 ? (R8 - (rb << 7)) : 128;
  return int64_t(rb) * 384 * Kt + int64_t(k >> 5) * 96 * h + (rr >> 3) * 768 + q * 256 + ((k & 31) >> 3) * 64 +
         (rr & 7) * 8 + (k & 7);
}
DMRG_HD inline int64_t blk_size(int R, int Kt) { return int64_t(3) * ((R + 7) & ~7) * Kt; }

// one K segment: A (M rows) and B (N rows) are blocked split matrices with the
// same K extent pad32(K); the MMA runs over k < K (elements past K are zero)
struct MixSeg {
  const uint16_t* A;
  const uint16_t* B;
  int K, pad;
};
// C (M x N) = alpha * sum_seg A_seg B_seg^T
//   mode 0: C stored as a float pair (hi, lo), row-major with ld = ldc, at Chi/Clo
//   mode 2: C is a blocked split matrix (R8 = crows, Kt = ldc) at Cp; tile row m
//           is its row row0 + m, tile column n its column n (N a multiple of 32)
//   mode 3: gathered rows (cm0 and M multiples of 8): the 8-row group g of A (one
//           8-row group of some blocked split matrix) is at A + bcol[2 u] +
//           s * bcol[2 u + 1] for K slab s, u = cm0 / 8 + g; row m is written,
//           scaled by acol[cm0 + m], into the row of the blocked split matrix C
//           whose row part (the terms of blk_off that depend on r) is
//           ccol[cm0 + m] & (2^48 - 1) and whose row block holds
//           8 * (ccol[cm0 + m] >> 48) rows (ccol < 0: padding, not stored)
struct MixProb {
  float* Chi;
  float* Clo;
  uint16_t* Cp;
  int ldc, M, N, s0, s1;
  float alpha;
  int mode, pad;
  int64_t cm0;
  int row0, crows;
};
// FP64 block (rows x cols, ld) -> blocked split matrices: element (r, c) goes to
// (rn0 + r, cn0 + c) of the matrix at dn (rn8 padded rows, K extent ktn) and/or
// to (rt0 + c, ct0 + r) of the matrix at dt (transposed copy)
struct SplitTask {
  const double* src;
  int rows, cols, ld;
  int rn0, cn0, rn8, ktn;
  int rt0, ct0, rt8, ktt;
  uint16_t* dn;
  uint16_t* dt;
};

class Exec {
 public:
  virtual ~Exec() {}
  virtual void* alloc(size_t bytes) = 0;
  // number of device allocations made so far (alloc calls, plan uploads included)
  virtual int64_t alloc_count() const = 0;
  virtual void release(void* p) = 0;
  virtual void zero(void* p, size_t bytes) = 0;
  virtual void h2d(void* d, const void* h, size_t bytes) = 0;
  // the same copy issued directly from h (no staging; allocates nothing)
  virtual void h2d_direct(void* d, const void* h, size_t bytes) = 0;
  virtual void d2h(void* h, const void* d, size_t bytes) = 0;
  virtual void d2d(void* d, const void* s, size_t bytes) = 0;
  virtual void sync() = 0;
  // stream-ordered timestamps: stamp() records an event on the stream and returns
  // its index; stamp_ms(a, b) = device milliseconds between two stamps (waits for
  // b); stamps_clear() synchronises the stream and releases them
  virtual int stamp() = 0;
  virtual double stamp_ms(int a, int b) = 0;
  virtual void stamps_clear() = 0;

  // grouped element-wise Kronecker accumulation (operator blocking)
  virtual void kron(const std::vector<KronGroup>& g, const std::vector<KronTask>& t) = 0;
  // grouped, segmented FP64 GEMM (one-shot upload)
  virtual void gemm(const std::vector<GemmProb>& p, const std::vector<GemmSeg>& s) = 0;
  // persistent plans (uploaded once, replayed during Davidson)
  virtual int gemm_plan(const std::vector<GemmProb>& p, const std::vector<GemmSeg>& s) = 0;
  virtual void gemm_run(int plan) = 0;
  virtual void plan_free(int plan) = 0;
  virtual void diag(const std::vector<DiagTask>& t) = 0;
  // generalised Fock matrix F_pq = sum_r t_pr g1_qr + sum_rst v_prst g2_qrst and the
  // orbital gradient grad_pq = 2 (F_qp - F_pq) (device arrays, row-major L x L / L^4)
  virtual void orbital_gradient(int L, const double* t, const double* v, const double* g1, const double* g2,
                                double* grad) = 0;
  // out[i] (device) = the Frobenius product of task i (fixed-order reductions)
  virtual void dots(const std::vector<DotTask>& t, double* out) = 0;

  // dense FP64 vector kernels on length-n vectors stored with a row stride
  // out[i*ldo + j] = sum_e V[i*ldv + e] * X[j*ldx + e]     (i < m, j < k)
  virtual void mdot(const double* V, int64_t ldv, int m, const double* X, int64_t ldx, int k,
                    int64_t n, double* out, int ldo) = 0;
  // Y_j = beta * Y_j + alpha * sum_i C[i*ldc + j] * V_i     (C is a device matrix)
  virtual void lincomb(const double* V, int64_t ldv, int m, const double* C, int ldc, int k,
                       int64_t n, double* Y, int64_t ldy, double alpha, double beta) = 0;
  // y += alpha * s[0] * x   (s is a device scalar)
  virtual void axpy_dev(const double* x, double* y, int64_t n, const double* s, double alpha) = 0;
  // t = r / (theta - diag), |theta - diag| floored at floor (theta device scalar)
  virtual void precond(const double* r, const double* diag, const double* theta, int64_t n,
                       double* t, double floor) = 0;
  // x *= 1 / sqrt(nrm2[0])
  virtual void normalize(double* x, int64_t n, const double* nrm2) = 0;
  // lowest eigenpair of the symmetric m x m matrix whose upper triangle is in H (ld ldh):
  // theta[0] = eigenvalue, y[0..m) = eigenvector
  virtual void ritz(const double* H, int ldh, int m, double* theta, double* y) = 0;
  // batched symmetric eigen-decomposition (Householder tridiagonalisation, divide
  // and conquer, FP64): A_b is n_b x n_b (ld = n_b, destroyed), w_b ascending
  // eigenvalues, Z_b eigenvectors as columns (ld n_b)
  virtual void syev(const std::vector<double*>& A, const std::vector<double*>& w,
                    const std::vector<double*>& Z, const std::vector<int>& n) = 0;

  // split-BF16 tensor-core GEMM plans (tcgen05 / TMEM)
  virtual int mix_plan(const std::vector<MixProb>& p, const std::vector<MixSeg>& s) = 0;
  // plan with the per-column tables of mode-3 problems
  virtual int mix_plan_g(const std::vector<MixProb>& p, const std::vector<MixSeg>& s,
                         const std::vector<int64_t>& bcol, const std::vector<int64_t>& ccol,
                         const std::vector<float>& acol) = 0;
  // the same with a tile schedule and shape: order 0 = longest tile first over the
  // whole list (the default), 1 = problems in the given order, each problem's tiles
  // together, 2 = problems by decreasing total work, each problem's tiles together;
  // width = tile width (MMA N) of every tile: 128 (the default), 64 or 32.  Every
  // choice computes each output element with the same products in the same order
  virtual int mix_plan_ordered(const std::vector<MixProb>& p, const std::vector<MixSeg>& s,
                               const std::vector<int64_t>& bcol, const std::vector<int64_t>& ccol,
                               const std::vector<float>& acol, int order, int width) = 0;
  virtual void mix_run(int plan) = 0;
  // milliseconds per run of a plan (CUDA events on the stream, after one warm-up run)
  virtual float mix_time(int plan, int reps) = 0;
  virtual void mix_plan_free(int plan) = 0;
  // host copy of a plan's problems, segments and gathered-row tables (kept so that
  // plans of several problems can be merged into one grouped launch)
  struct MixPlanHost {
    std::vector<MixProb> p;
    std::vector<MixSeg> s;
    std::vector<int64_t> bcol, ccol;
    std::vector<float> acol;
  };
  virtual const MixPlanHost& mix_plan_host(int plan) const = 0;
  // the CUDA stream (cudaStream_t) all work is ordered on, and whether kernel
  // timing is on (timing records events and drains them with host waits)
  virtual void* stream() const = 0;
  virtual bool profiling() const = 0;
  // CUDA graphs of this executor's work: capture(f) records the work f issues on the
  // stream into an instantiated graph (-1 when the stream cannot be captured: the
  // default stream, or kernel timing on); graph_run replays it on the stream
  virtual int graph_capture(const std::function<void()>& f) = 0;
  virtual void graph_run(int id) = 0;
  virtual void graph_free(int id) = 0;
  virtual int split_plan(const std::vector<SplitTask>& t) = 0;
  virtual void split_run(int plan) = 0;
  virtual void split_plan_free(int plan) = 0;
  virtual void df_to_f64(const float* hi, const float* lo, double* out, int64_t n) = 0;
  // (hi, lo)[i] (+)= sum_q part[q] (double-float pairs: part + q*2n holds n hi then n lo)
  virtual void reduce_parts(const float* part, int nparts, int64_t n, float* hi, float* lo, int accumulate) = 0;
  // nonzero when a bounded device-side wait gave up (read with a stream sync)
  virtual int device_error() = 0;

  // kernel timing with events on the stream: mode 1 resets and starts, mode 0 stops
  // and fills out[2*c] = milliseconds, out[2*c+1] = launches for each kernel class c
  // (0 gemm_f64, 1 kron, 2 vector, 3 syev/ritz, 4 mixed gemm stage 2 / accumulate,
  //  5 split/pack/reduce, 6 mixed gemm stage 1 (BF16-plane output))
  virtual void profile(int mode, double* out) = 0;
};

enum { PROF_GEMM = 0, PROF_KRON, PROF_VEC, PROF_EIG, PROF_MIXED, PROF_SPLIT, PROF_MIXED1, PROF_N };

Exec* make_cuda_exec(void* stream, int precision_mode);

}  // namespace dmrg
