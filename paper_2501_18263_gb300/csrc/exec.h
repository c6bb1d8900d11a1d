// Numerical primitives the DMRG host core drives.  The product library
// implements them with sm_103a kernels (exec_cuda.cu); every pointer handed to
// them is a device pointer owned by the engine's arenas.
#pragma once
#include <cstddef>
#include <cstdint>
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

// ---- split-BF16 tensor-core path -------------------------------------------
// Operands are stored as three BF16 planes (x ~ hi + mid + lo), plane p of an
// operand at ptr + p * plane_stride.  Every operand is K-major: row r holds K
// contiguous elements at ptr + r * ld; rows start on 16-byte boundaries (ld and
// plane strides multiples of 8 elements) and the elements between K and
// round8(K) are zero.
struct MixSeg {
  const uint16_t* A;   // M rows (tile rows) x K
  const uint16_t* B;   // N rows (tile cols) x K
  int64_t psA, psB;
  int lda, ldb, K, pad;
};
// C (M x N) = alpha * sum_seg A_seg B_seg^T
//   mode 0: C kept as a float pair (hi, lo) at Chi/Clo (+= if accumulate)
//   mode 1: C written as three BF16 planes at Cp (plane stride psC)
//   mode 2: as mode 1 but transposed: tile column n is written to row n of C
//   mode 3: gathered columns: column n takes its B row at B + bcol[cm0 + n] and is
//           written (transposed, scaled by acol[cm0 + n]) to Cp + ccol[cm0 + n]
struct MixProb {
  float* Chi;
  float* Clo;
  uint16_t* Cp;
  int64_t psC;
  int ldc, M, N, s0, s1;
  float alpha;
  int mode, accumulate;
  int64_t cm0;
};
// FP64 block (rows x cols, ld) -> BF16 planes, normal (rows x ldn) and/or transposed (cols x ldt)
struct SplitTask {
  const double* src;
  int rows, cols, ld, ldn, ldt, pad;
  uint16_t* dn;
  uint16_t* dt;
  int64_t ps;
};

class Exec {
 public:
  virtual ~Exec() {}
  virtual void* alloc(size_t bytes) = 0;
  virtual void release(void* p) = 0;
  virtual void zero(void* p, size_t bytes) = 0;
  virtual void h2d(void* d, const void* h, size_t bytes) = 0;
  virtual void d2h(void* h, const void* d, size_t bytes) = 0;
  virtual void d2d(void* d, const void* s, size_t bytes) = 0;
  virtual void sync() = 0;

  // grouped element-wise Kronecker accumulation (operator blocking)
  virtual void kron(const std::vector<KronGroup>& g, const std::vector<KronTask>& t) = 0;
  // grouped, segmented FP64 GEMM (one-shot upload)
  virtual void gemm(const std::vector<GemmProb>& p, const std::vector<GemmSeg>& s) = 0;
  // persistent plans (uploaded once, replayed during Davidson)
  virtual int gemm_plan(const std::vector<GemmProb>& p, const std::vector<GemmSeg>& s) = 0;
  virtual void gemm_run(int plan) = 0;
  virtual void plan_free(int plan) = 0;
  virtual void diag(const std::vector<DiagTask>& t) = 0;

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
  // batched symmetric eigen-decomposition (cyclic Jacobi, FP64): A_b is n_b x n_b
  // (ld = n_b, destroyed), w_b ascending eigenvalues, Z_b eigenvectors as columns (ld n_b)
  virtual void syev(const std::vector<double*>& A, const std::vector<double*>& w,
                    const std::vector<double*>& Z, const std::vector<int>& n) = 0;

  // split-BF16 tensor-core GEMM plans (tcgen05 / TMEM)
  virtual int mix_plan(const std::vector<MixProb>& p, const std::vector<MixSeg>& s) = 0;
  // plan with the per-column tables of mode-3 problems
  virtual int mix_plan_g(const std::vector<MixProb>& p, const std::vector<MixSeg>& s,
                         const std::vector<int64_t>& bcol, const std::vector<int64_t>& ccol,
                         const std::vector<float>& acol) = 0;
  virtual void mix_run(int plan) = 0;
  virtual void mix_plan_free(int plan) = 0;
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
