// CUDA executor: the sm_103a kernels behind the host core's numerical steps.
//   gemm_f64      grouped, segmented FP64 GEMM (the FP64 sigma / Ren / StVec path)
//   kron          grouped Kronecker accumulation (operator blocking)
//   mdot/lincomb  Davidson Gram-Schmidt and Ritz vectors (deterministic reductions)
//   ritz          cyclic Jacobi eigensolver of the small Rayleigh-Ritz matrix
//   syev          density-matrix eigensolver of the truncation: Householder
//                 tridiagonalisation (a CTA cluster per large sector block), divide
//                 and conquer on the tridiagonal matrices (tridiag_dc.cu), W = Q V
// All work is ordered on one stream; allocations are stream-ordered.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../exec.h"
#include "../exec_errors.h"
#include "mixed.h"
#include "tridiag_dc.h"

namespace dmrg {

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      if (e_ == cudaErrorMemoryAllocation) throw OomError(std::string("CUDA: ") + cudaGetErrorString(e_)); \
      throw CudaError(std::string(#x) + ": " + cudaGetErrorString(e_));               \
    }                                                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// grouped FP64 GEMM: one CTA per 64 x 64 output tile, K loop over all segments

struct GemmTile {
  int prob, m0, n0, pad;
};

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmTile* __restrict__ tiles,
                                                       const GemmProb* __restrict__ probs,
                                                       const GemmSeg* __restrict__ segs) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmProb p = probs[tl.prob];
  const int tid = threadIdx.x;
  // warp w owns rows 16 (w / 2) .. +15 and columns 32 (w % 2) .. +31 of the
  // tile, its lanes 4 x 8 sub-tiles of 4 x 4; a warp whose rows or columns lie
  // wholly past a ragged edge skips the multiply-adds (warp-uniform test)
  const int warp = tid >> 5, lane = tid & 31;
  const int ty = 4 * (warp >> 1) + (lane >> 3), tx = 8 * (warp & 1) + (lane & 7);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int Mt = min(TM, p.M - tl.m0), Nt = min(TN, p.N - tl.n0);
  const bool busy = 16 * (warp >> 1) < Mt && 32 * (warp & 1) < Nt;
  for (int s = p.s0; s < p.s1; ++s) {
    const GemmSeg g = segs[s];
    for (int k0 = 0; k0 < g.K; k0 += TK) {
      const int Kt = min(TK, g.K - k0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = tid + 256 * r;
        int m, k;
        if (g.ta == 0) { m = i >> 4; k = i & 15; } else { m = i & 63; k = i >> 6; }
        double a = 0.0;
        if (m < Mt && k < Kt) {
          const int64_t gm = tl.m0 + m, gk = k0 + k;
          a = g.ta == 0 ? g.A[gm * g.lda + gk] : g.A[gk * g.lda + gm];
        }
        As[k][m] = a;
        int n, kb;
        if (g.tb == 0) { n = i & 63; kb = i >> 6; } else { n = i >> 4; kb = i & 15; }
        double b = 0.0;
        if (n < Nt && kb < Kt) {
          const int64_t gn = tl.n0 + n, gk = k0 + kb;
          b = g.tb == 0 ? g.B[gk * g.ldb + gn] : g.B[gn * g.ldb + gk];
        }
        Bs[kb][n] = b;
      }
      __syncthreads();
      if (busy) {
        // a ragged K step (Kt < TK: the last one of a segment) runs only its own k
#pragma unroll 4
        for (int k = 0; k < Kt; ++k) {
          double a[4], b[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
          for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = ty * 4 + i;
    if (m >= Mt) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = tx * 4 + j;
      if (n >= Nt) continue;
      double* c = p.C + int64_t(tl.m0 + m) * p.ldc + tl.n0 + n;
      const double v = p.alpha * acc[i][j];
      *c = p.accumulate ? *c + v : v;
    }
  }
}

// ---------------------------------------------------------------------------
// grouped Kronecker accumulation

constexpr int KRON_CHUNK = 1024;   // elements of one group per CTA

// CTA base + b works on chunk base + b - cpre[k] of the group k with
// cpre[k] <= base + b < cpre[k + 1] (prefix sums of the groups' chunk counts), so
// the host lists groups only, not CTAs
__global__ void __launch_bounds__(256) kron_kernel(const int64_t* __restrict__ cpre, int ngroups, int64_t base,
                                                   const KronGroup* __restrict__ groups,
                                                   const KronTask* __restrict__ tasks) {
  const int64_t cb = base + blockIdx.x;
  int lo = 0, hi = ngroups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cpre[mid] <= cb) lo = mid;
    else hi = mid - 1;
  }
  const KronGroup g = groups[lo];
  const int n = g.rows * g.cols;
  const int e0 = int((cb - cpre[lo]) * KRON_CHUNK);
  const int e1 = min(n, e0 + KRON_CHUNK);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int r = e / g.cols, col = e - r * g.cols;
    double acc = 0.0;
    for (int t = g.t0; t < g.t1; ++t) {
      const KronTask k = tasks[t];
      double v;
      if (k.mode == 0) v = k.src[int64_t(r) * k.src_ld + col];
      else if (k.mode == 1) v = k.src[int64_t(col) * k.src_ld + r];
      else v = (r == col) ? 1.0 : 0.0;
      acc = fma(k.coef, v, acc);
    }
    double* d = g.dst + int64_t(r) * g.ld + col;
    *d = g.accumulate ? *d + acc : acc;
  }
}

// one CTA per task (grid-stride), each thread a fixed subset of the elements, then a
// fixed warp / block tree: the result does not depend on scheduling
__global__ void __launch_bounds__(128) dot_tasks_kernel(const DotTask* __restrict__ t, int nt,
                                                        double* __restrict__ out) {
  __shared__ double red[4];
  for (int i = blockIdx.x; i < nt; i += gridDim.x) {
    const DotTask d = t[i];
    const int n = d.rows * d.cols;
    double acc = 0.0;
    if (d.mode == 2) {
      for (int r = threadIdx.x; r < min(d.rows, d.cols); r += blockDim.x) acc += d.a[int64_t(r) * d.lda + r];
    } else {
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int r = e / d.cols, c = e - r * d.cols;
        const double bv = d.mode == 0 ? d.b[int64_t(r) * d.ldb + c] : d.b[int64_t(c) * d.ldb + r];
        acc = fma(d.a[int64_t(r) * d.lda + c], bv, acc);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) out[i] = (red[0] + red[1]) + (red[2] + red[3]);
    __syncthreads();
  }
}

// F_pq = sum_r t_pr g1_qr + sum_rst v_prst g2_qrst: one CTA per (p, q), the two
// contiguous rows t[p, :] . g1[q, :] and v[p, ...] . g2[q, ...] (L + L^3 products)
__global__ void __launch_bounds__(128) fock_kernel(int L, const double* __restrict__ t, const double* __restrict__ v,
                                                   const double* __restrict__ g1, const double* __restrict__ g2,
                                                   double* __restrict__ F) {
  __shared__ double red[4];
  const int p = blockIdx.x / L, q = blockIdx.x % L;
  const int64_t L3 = int64_t(L) * L * L;
  double acc = 0.0;
  for (int r = threadIdx.x; r < L; r += blockDim.x) acc = fma(t[int64_t(p) * L + r], g1[int64_t(q) * L + r], acc);
  const double* vp = v + p * L3;
  const double* gq = g2 + q * L3;
  for (int64_t e = threadIdx.x; e < L3; e += blockDim.x) acc = fma(vp[e], gq[e], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) F[blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
}

__global__ void orbital_grad_kernel(int L, const double* __restrict__ F, double* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L * L) return;
  const int p = i / L, q = i % L;
  g[i] = 2.0 * (F[q * L + p] - F[p * L + q]);
}

__global__ void diag_kernel(const DiagTask* __restrict__ t, int nt) {
  for (int i = blockIdx.x; i < nt; i += gridDim.x) {
    const DiagTask d = t[i];
    for (int e = threadIdx.x; e < d.n; e += blockDim.x)
      d.dst[e * d.dst_stride] = d.coef * (d.src ? d.src[int64_t(e) * (d.ld + 1)] : 1.0);
  }
}

// ---------------------------------------------------------------------------
// vector kernels

constexpr int MDOT_MAX = 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) mdot_partial(const double* __restrict__ V, int64_t ldv, int m,
                                                    const double* __restrict__ X, int64_t ldx, int64_t n,
                                                    double* __restrict__ part) {
  const int j = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
  const int64_t e0 = n * b / nb, e1 = n * (b + 1) / nb;
  double acc[MDOT_MAX];
#pragma unroll
  for (int i = 0; i < MDOT_MAX; ++i) acc[i] = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double x = X[j * ldx + e];
#pragma unroll
    for (int i = 0; i < MDOT_MAX; ++i)
      if (i < m) acc[i] = fma(V[i * ldv + e], x, acc[i]);
  }
  __shared__ double red[8][MDOT_MAX];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MDOT_MAX; ++i) {
    if (i >= m) break;
    double s = warp_sum(acc[i]);
    if (l == 0) red[w][i] = s;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    double s = 0.0;
    for (int ww = 0; ww < 8; ++ww) s += red[ww][threadIdx.x];
    part[(int64_t(b) * gridDim.y + j) * MDOT_MAX + threadIdx.x] = s;
  }
}

__global__ void mdot_final(const double* __restrict__ part, int nb, int m, int k, double* out, int ldo) {
  const int t = threadIdx.x + blockIdx.x * blockDim.x;
  if (t >= m * k) return;
  const int i = t / k, j = t % k;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t(b) * k + j) * MDOT_MAX + i];
  out[i * ldo + j] = s;
}

__global__ void lincomb_kernel(const double* __restrict__ V, int64_t ldv, int m, const double* __restrict__ C,
                               int ldc, int k, int64_t n, double* Y, int64_t ldy, double alpha, double beta) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s = fma(C[i * ldc + j], V[i * ldv + e], s);
      double* y = Y + j * ldy + e;
      *y = (beta == 0.0 ? 0.0 : beta * *y) + alpha * s;
    }
}

__global__ void axpy_dev_kernel(const double* __restrict__ x, double* y, int64_t n, const double* s, double alpha) {
  const double a = alpha * s[0];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    y[e] = fma(a, x[e], y[e]);
}

__global__ void precond_kernel(const double* __restrict__ r, const double* __restrict__ d, const double* th,
                               int64_t n, double* t, double fl) {
  const double theta = th[0];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    double den = theta - d[e];
    if (fabs(den) < fl) den = den < 0 ? -fl : fl;
    t[e] = r[e] / den;
  }
}

__global__ void normalize_kernel(double* x, int64_t n, const double* nrm2) {
  const double s = 1.0 / sqrt(nrm2[0]);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    x[e] *= s;
}

// ---------------------------------------------------------------------------
// cyclic Jacobi with the round-robin (tournament) pair ordering: n/2 disjoint
// rotations per step are computed from the current matrix and applied together.

template <bool SHARED>
__device__ void jacobi_core(double* A, double* Z, int n, int ld, double* cs, int* pp, int* qq, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = n + (n & 1);  // even count (dummy index ne-1 when n is odd)
  for (int e = tid; e < n * n; e += nt) Z[(e / n) * ld + e % n] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    // convergence: off-diagonal Frobenius norm relative to the full norm
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      const double a = A[i * ld + j];
      tot += a * a;
      if (i != j) off += a * a;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = off;
      red[2 * (tid >> 5) + 1] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      double o = 0, t = 0;
      for (int w = 0; w < nt / 32; ++w) {
        o += red[2 * w];
        t += red[2 * w + 1];
      }
      red[64] = (o <= 1e-26 * t || t == 0.0) ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool done = red[64] != 0.0;
    __syncthreads();
    if (done) break;
    for (int step = 0; step < ne - 1; ++step) {
      // pairs of the round-robin schedule
      for (int k = tid; k < ne / 2; k += nt) {
        int a, b;
        if (k == 0) {
          a = ne - 1;
          b = step;
        } else {
          a = (step + k) % (ne - 1);
          b = (step - k + ne - 1) % (ne - 1);
        }
        int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * ld + q];
          if (apq != 0.0) {
            const double app = A[p * ld + p], aqq = A[q * ld + q];
            const double th = (aqq - app) / (2.0 * apq);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pp[k] = p;
        qq[k] = q;
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // columns: A <- A J, Z <- Z J
      for (int e = tid; e < (ne / 2) * n; e += nt) {
        const int k = e / n, row = e % n;
        const int p = pp[k], q = qq[k];
        if (q >= n) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        if (s == 0.0) continue;
        const double ap = A[row * ld + p], aq = A[row * ld + q];
        A[row * ld + p] = c * ap - s * aq;
        A[row * ld + q] = s * ap + c * aq;
        const double zp = Z[row * ld + p], zq = Z[row * ld + q];
        Z[row * ld + p] = c * zp - s * zq;
        Z[row * ld + q] = s * zp + c * zq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < (ne / 2) * n; e += nt) {
        const int k = e / n, col = e % n;
        const int p = pp[k], q = qq[k];
        if (q >= n) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        if (s == 0.0) continue;
        const double ap = A[p * ld + col], aq = A[q * ld + col];
        A[p * ld + col] = c * ap - s * aq;
        A[q * ld + col] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
}

// Batched symmetric eigen-decomposition A = Z diag(w) Z^T (FP64) in phases that
// each spread over the GPU (FP64 on this GPU issues one instruction per warp every
// few tens of cycles, so a sequential recurrence on one thread, such as the QL
// iteration's chain of plane rotations, would dominate):
//  1. Householder reduction to tridiagonal form, A = Q T Q^T with
//     Q = H_0 ... H_{n-3}, H_k = I - tau_k u_k u_k^T (u_k supported on k+1..n-1),
//     one CTA per small matrix, a cluster of eight per large one (syev_tridiag_kernel);
//  2. Q formed explicitly, one warp per column: column j of Q is e_j with the
//     reflectors k < j applied in the order k = j-1, ..., 0 (the reflectors k >= j
//     leave e_j alone) (syev_qform_kernel);
//  3. T = V diag(w) V^T by divide and conquer (tridiag_dc.cu: leaves of at most 32
//     rows by implicit QL on one warp, merges level by level over all matrices);
//  4. W = Q V, a grouped FP64 GEMM;
//  5. eigenvalues sorted ascending, eigenvectors permuted with them
//     (syev_sort_kernel, syev_perm_kernel).
struct SyevJob {
  double* A;      // n x n input, destroyed; then V, the eigenvectors of T (column-major)
  double* w;      // out: n eigenvalues, ascending
  double* Z;      // out: n x n eigenvectors as columns (row-major, ld n)
  double* d;      // n: diagonal of T, then the (unsorted) eigenvalues
  double* e;      // n: off-diagonal of T (e[i] couples i and i + 1)
  double* tau;    // n: reflector scalars
  double* Zc;     // n x n, column-major (Zc[c * n + r]): Q
  double* U;      // n x n: reflector k in row k (u_k[k + 1] = 1), then W = Q V (column-major)
  double* pb;     // n: p = tau A22 v exchanged between the CTAs of a cluster
  int* perm;      // n: sorted position of eigenvalue i
  int n, pad;
};

constexpr int SYEV_THREADS = 1024;
constexpr int SYEV_CLUSTER = 8;   // CTAs per large matrix in the reduction (portable cluster size)

// sum over the CTA, returned to every thread (red: >= 33 doubles of shared memory)
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = lane < int(blockDim.x >> 5) ? red[lane] : 0.0;
    x = warp_sum(x);
    if (lane == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}

// index j of the segment holding x, given prefix sums pre[0..nj] (pre[0] = 0)
__device__ __forceinline__ int syev_find(const int* pre, int nj, int x) {
  int lo = 0, hi = nj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// step 1: a cluster of CS CTAs per matrix (CS = 1: one CTA).  Per column k every
// CTA reads row k and forms the same reflector (the same reductions in the same
// order); the rows of the trailing block are dealt out warp by warp over the
// cluster for p = tau A22 v and for the rank-2 update, p is exchanged through
// global scratch, and two cluster barriers per column order the steps (p complete
// before it is read; the update complete before row k + 1 is read and before p is
// overwritten).  The reflector goes to U (row k), so no CTA writes a row another
// may still be reading.
__device__ __forceinline__ uint32_t syev_cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void syev_cluster_sync() {
  __threadfence();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int CS>
__global__ void __launch_bounds__(SYEV_THREADS) syev_tridiag_kernel(const SyevJob* jobs, const int* sel, int maxn) {
  const int rank = CS > 1 ? int(syev_cluster_rank()) : 0;
  const SyevJob jb = jobs[sel[blockIdx.x / CS]];
  const int n = jb.n;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  extern __shared__ double sm[];
  double* vs = sm;             // Householder vector of the current step
  double* ps = vs + maxn;      // p = tau A22 v, then w
  double* red = ps + maxn;     // 40 doubles: reductions and scalars
  double* A = jb.A;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const double* x = A + int64_t(k) * n + k + 1;    // row k right of the diagonal (= column k below it)
    double part = 0.0;
    for (int i = 1 + tid; i < m; i += nt) part += x[i] * x[i];
    const double sigma = block_sum(part, red);
    if (tid == 0) {
      const double alpha = x[0];
      double beta = alpha, tau = 0.0, scale = 0.0;
      if (sigma != 0.0) {
        const double mu = sqrt(alpha * alpha + sigma);
        beta = alpha <= 0.0 ? mu : -mu;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      red[34] = scale;
      red[35] = tau;
      if (rank == 0) {
        jb.d[k] = A[int64_t(k) * n + k];
        jb.e[k] = beta;
        jb.tau[k] = tau;
      }
    }
    __syncthreads();
    const double tau = red[35], scale = red[34];
    if (tau == 0.0) continue;   // H_k = I: A unchanged
    double* u = jb.U + int64_t(k) * n + k + 1;
    for (int i = tid; i < m; i += nt) {
      const double v = i == 0 ? 1.0 : x[i] * scale;
      vs[i] = v;
      if (rank == 0) u[i] = v;   // the reflector, for step 2
    }
    __syncthreads();
    // p = tau A22 v: one warp per row, rows dealt out over the cluster's warps
    double* A22 = A + int64_t(k + 1) * n + k + 1;
    for (int r = rank * nw + wid; r < m; r += CS * nw) {
      const double* row = A22 + int64_t(r) * n;
      double acc = 0.0;
      for (int j = lane; j < m; j += 32) acc += row[j] * vs[j];
      acc = warp_sum(acc);
      if (lane == 0) {
        if (CS > 1) jb.pb[r] = tau * acc;
        else ps[r] = tau * acc;
      }
    }
    if (CS > 1) {
      syev_cluster_sync();
      for (int i = tid; i < m; i += nt) ps[i] = jb.pb[i];
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = tid; i < m; i += nt) pv += ps[i] * vs[i];
    const double K = 0.5 * tau * block_sum(pv, red);
    for (int i = tid; i < m; i += nt) ps[i] -= K * vs[i];   // w
    __syncthreads();
    // A22 -= v w^T + w v^T on the same rows
    for (int r = rank * nw + wid; r < m; r += CS * nw) {
      double* row = A22 + int64_t(r) * n;
      const double vr = vs[r], wr = ps[r];
      for (int j = lane; j < m; j += 32) row[j] -= vr * ps[j] + wr * vs[j];
    }
    if (CS > 1) syev_cluster_sync();
    else __syncthreads();
  }
  if (tid == 0 && rank == 0) {
    if (n >= 2) {
      jb.d[n - 2] = A[int64_t(n - 2) * n + n - 2];
      jb.e[n - 2] = A[int64_t(n - 2) * n + n - 1];
    }
    jb.d[n - 1] = A[int64_t(n - 1) * n + n - 1];
    jb.e[n - 1] = 0.0;
  }
}

// step 2: one warp per column of Q (pre: prefix sums of the matrices' n)
__global__ void __launch_bounds__(256) syev_qform_kernel(const SyevJob* jobs, const int* pre, int nj) {
  const int gw = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (gw >= pre[nj]) return;
  const int b = syev_find(pre, nj, gw);
  const SyevJob jb = jobs[b];
  const int n = jb.n, j = gw - pre[b];
  double* z = jb.Zc + int64_t(j) * n;
  for (int i = lane; i < n; i += 32) z[i] = (i == j) ? 1.0 : 0.0;
  __syncwarp();
  for (int k = min(j - 1, n - 3); k >= 0; --k) {
    const double tau = jb.tau[k];
    if (tau == 0.0) continue;
    const int m = n - k - 1;
    const double* u = jb.U + int64_t(k) * n + k + 1;   // u[0] = 1
    double* zz = z + k + 1;
    double acc = 0.0;
    for (int i = lane; i < m; i += 32) acc += u[i] * zz[i];
    acc = tau * warp_sum(acc);
    for (int i = lane; i < m; i += 32) zz[i] -= acc * u[i];
    __syncwarp();
  }
}

// step 5a: rank of every eigenvalue (ties by index); w in ascending order
__global__ void __launch_bounds__(256) syev_sort_kernel(const SyevJob* jobs, const int* pre, int nj) {
  const int g = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= pre[nj]) return;
  const int b = syev_find(pre, nj, g);
  const SyevJob jb = jobs[b];
  const int i = g - pre[b];
  const double di = jb.d[i];
  int r = 0;
  for (int j = 0; j < jb.n; ++j) {
    const double dj = jb.d[j];
    r += (dj < di) || (dj == di && j < i);
  }
  jb.w[r] = di;
  jb.perm[i] = r;
}

// step 5b: one CTA per eigenvector: column i of Zc to column perm[i] of Z
__global__ void __launch_bounds__(128) syev_perm_kernel(const SyevJob* jobs, const int* pre, int nj) {
  const int g = int(blockIdx.x);
  const int b = syev_find(pre, nj, g);
  const SyevJob jb = jobs[b];
  const int n = jb.n, i = g - pre[b];
  const int to = jb.perm[i];
  const double* src = jb.U + int64_t(i) * n;   // W = Q V
  for (int row = threadIdx.x; row < n; row += blockDim.x) jb.Z[int64_t(row) * n + to] = src[row];
}

// Rayleigh-Ritz of the Davidson subspace: lowest eigenpair of an m x m matrix (m <= 40)
__global__ void __launch_bounds__(64) ritz_kernel(const double* H, int ldh, int m, double* theta, double* y) {
  __shared__ double A[40 * 40];
  __shared__ double Z[40 * 40];
  __shared__ double cs[44];
  __shared__ double red[72];
  __shared__ int pp[22], qq[22];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    A[i * m + j] = i <= j ? H[i * ldh + j] : H[j * ldh + i];
  }
  __syncthreads();
  jacobi_core<true>(A, Z, m, m, cs, pp, qq, red);
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int i = 1; i < m; ++i)
      if (A[i * m + i] < A[best * m + best]) best = i;
    theta[0] = A[best * m + best];
    // fix the sign: largest-magnitude component positive
    int arg = 0;
    for (int i = 1; i < m; ++i)
      if (fabs(Z[i * m + best]) > fabs(Z[arg * m + best])) arg = i;
    const double sg = Z[arg * m + best] < 0 ? -1.0 : 1.0;
    for (int i = 0; i < m; ++i) y[i] = sg * Z[i * m + best];
  }
}

// ---------------------------------------------------------------------------

class CudaExec : public Exec {
  struct Mark {
    cudaEvent_t a, b;
    int cls;
  };
  bool prof_ = false;
  std::vector<Mark> marks_;
  std::vector<cudaEvent_t> pool_;
  std::vector<cudaEvent_t> stamps_;   // phase timestamps (stamp)
  double acc_[2 * PROF_N] = {};
  cudaEvent_t ev() {
    if (pool_.empty()) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = pool_.back();
    pool_.pop_back();
    return e;
  }
  // bracket one launch with events when profiling
  template <class F>
  void launch(int cls, F&& f) {
    if (!prof_) {
      f();
      CK(cudaGetLastError());
      return;
    }
    Mark m{ev(), ev(), cls};
    CK(cudaEventRecord(m.a, st_));
    f();
    CK(cudaGetLastError());
    CK(cudaEventRecord(m.b, st_));
    marks_.push_back(m);
    if (marks_.size() > 4096) drain();
  }
  void drain() {
    if (marks_.empty()) return;
    CK(cudaEventSynchronize(marks_.back().b));
    for (auto& m : marks_) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, m.a, m.b));
      acc_[2 * m.cls] += ms;
      acc_[2 * m.cls + 1] += 1;
      pool_.push_back(m.a);
      pool_.push_back(m.b);
    }
    marks_.clear();
  }

 public:
  void profile(int mode, double* out) override {
    if (mode == 1) {
      drain();
      for (double& x : acc_) x = 0;
      prof_ = true;
    } else {
      drain();
      prof_ = false;
      if (out)
        for (int i = 0; i < 2 * PROF_N; ++i) out[i] = acc_[i];
    }
  }

  CudaExec(void* stream, int prec) : st_(static_cast<cudaStream_t>(stream)), prec_(prec) {
    CK(cudaGetDevice(&dev_));
    CK(cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev_));
    CK(cudaMalloc(&part_, sizeof(double) * 1024 * MDOT_MAX * 4));
    CK(cudaMalloc(&err_, sizeof(int)));
    CK(cudaMemsetAsync(err_, 0, sizeof(int), st_));
    // stream-ordered allocations come from the device's default pool, which by
    // default returns freed memory to the system at every synchronisation, so that
    // each sweep step would map its multi-gigabyte arenas afresh: keep up to a
    // quarter of the device memory cached while a handle lives (trimmed when it
    // goes away; a process-local pool attribute)
    CK(cudaDeviceGetDefaultMemPool(&mpool_, dev_));
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    uint64_t thr = 0;
    CK(cudaMemPoolGetAttribute(mpool_, cudaMemPoolAttrReleaseThreshold, &thr));
    if (thr < tot / 4) {
      thr = tot / 4;
      CK(cudaMemPoolSetAttribute(mpool_, cudaMemPoolAttrReleaseThreshold, &thr));
    }
  }
  ~CudaExec() override {
    for (auto& g : graphs_)
      if (g) cudaGraphExecDestroy(g);
    try { drain(); } catch (...) {}
    for (auto& m : marks_) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (auto e : stamps_) cudaEventDestroy(e);
    for (auto e : pool_) cudaEventDestroy(e);
    for (auto& p : plans_) free_plan_mem(p);
    for (size_t i = 0; i < mplans_.size(); ++i) mix_free(int(i));
    for (auto& p : splans_)
      if (p.live) cudaFreeAsync(p.t, st_);
    cudaStreamSynchronize(st_);
    cudaFree(part_);
    cudaFree(err_);
    if (stage_ev_) cudaEventDestroy(stage_ev_);
    if (stage_) cudaFreeHost(stage_);
    if (mpool_) cudaMemPoolTrimTo(mpool_, 0);
  }
  int64_t alloc_count() const override { return n_alloc_; }
  void* alloc(size_t b) override {
    void* p = nullptr;
    ++n_alloc_;
    cudaError_t e = cudaMallocAsync(&p, b ? b : 8, st_);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw OomError("device allocation of " + std::to_string(b) + " bytes failed: " + cudaGetErrorString(e));
    }
    return p;
  }
  void release(void* p) override {
    if (p) CK(cudaFreeAsync(p, st_));
  }
  void zero(void* p, size_t b) override {
    if (b) CK(cudaMemsetAsync(p, 0, b, st_));
  }
  void h2d_direct(void* d, const void* h, size_t b) override {
    if (b) CK(cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, st_));
  }
  // Host-to-device copies go through a pinned staging ring: a copy from pageable
  // memory first waits for all work queued on the stream, so every plan upload
  // would stall the host until the GPU caught up.  The ring is filled front to
  // back; an event recorded after each staged copy marks how far the device has
  // read it, and the host waits on that event only when the ring wraps (the
  // stream runs in order, so the last copy done means every earlier one is).
  // Copies during stream capture, or larger than the ring may grow to, go direct.
  void h2d(void* d, const void* h, size_t b) override {
    if (!b) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st_, &cs));
    const size_t need = (b + 255) & ~size_t(255);
    if (cs != cudaStreamCaptureStatusNone || need > kStageMax / 2) {
      CK(cudaMemcpyAsync(d, h, b, cudaMemcpyHostToDevice, st_));
      return;
    }
    if (!stage_ev_) CK(cudaEventCreateWithFlags(&stage_ev_, cudaEventDisableTiming));
    if (2 * need > stage_cap_) {   // grow (after the device has read what is staged)
      size_t cap = std::max<size_t>(stage_cap_ ? stage_cap_ : (size_t(32) << 20), 2 * need);
      cap = std::min(cap, kStageMax);
      if (stage_) {
        CK(cudaEventSynchronize(stage_ev_));
        CK(cudaFreeHost(stage_));
        stage_ = nullptr;
      }
      CK(cudaHostAlloc(reinterpret_cast<void**>(&stage_), cap, cudaHostAllocDefault));
      stage_cap_ = cap;
      stage_head_ = 0;
    } else if (stage_head_ + need > stage_cap_) {
      CK(cudaEventSynchronize(stage_ev_));
      stage_head_ = 0;
    }
    char* src = stage_ + stage_head_;
    stage_head_ += need;
    std::memcpy(src, h, b);
    CK(cudaMemcpyAsync(d, src, b, cudaMemcpyHostToDevice, st_));
    CK(cudaEventRecord(stage_ev_, st_));
  }
  void d2h(void* h, const void* d, size_t b) override {
    if (b) {
      CK(cudaMemcpyAsync(h, d, b, cudaMemcpyDeviceToHost, st_));
      CK(cudaStreamSynchronize(st_));
    }
  }
  void d2d(void* d, const void* s, size_t b) override {
    if (b && d != s) CK(cudaMemcpyAsync(d, s, b, cudaMemcpyDeviceToDevice, st_));
  }
  void sync() override { CK(cudaStreamSynchronize(st_)); }
  int stamp() override {
    cudaEvent_t e = ev();
    stamps_.push_back(e);
    CK(cudaEventRecord(e, st_));
    return int(stamps_.size() - 1);
  }
  double stamp_ms(int a, int b) override {
    CK(cudaEventSynchronize(stamps_.at(size_t(b))));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, stamps_.at(size_t(a)), stamps_.at(size_t(b))));
    return double(ms);
  }
  void stamps_clear() override {
    CK(cudaStreamSynchronize(st_));
    for (cudaEvent_t e : stamps_) pool_.push_back(e);
    stamps_.clear();
  }

  template <class T>
  T* upload(const std::vector<T>& v) {
    T* d = static_cast<T*>(alloc(sizeof(T) * std::max<size_t>(v.size(), 1)));
    h2d(d, v.data(), sizeof(T) * v.size());
    return d;
  }

  void kron(const std::vector<KronGroup>& g, const std::vector<KronTask>& t) override {
    if (g.empty()) return;
    if (g.size() > size_t(INT32_MAX)) throw std::runtime_error("kron: too many groups");
    std::vector<int64_t> cpre(g.size() + 1, 0);
    for (size_t i = 0; i < g.size(); ++i)
      cpre[i + 1] = cpre[i] + (int64_t(g[i].rows) * g[i].cols + KRON_CHUNK - 1) / KRON_CHUNK;
    const int64_t nct = cpre.back();
    KronGroup* dg = upload(g);
    KronTask* dt = upload(t);
    int64_t* dc = upload(cpre);
    for (int64_t c0 = 0; c0 < nct; c0 += (int64_t(1) << 30)) {
      const unsigned nb = unsigned(std::min<int64_t>(nct - c0, int64_t(1) << 30));
      launch(PROF_KRON, [&] { kron_kernel<<<nb, 256, 0, st_>>>(dc, int(g.size()), c0, dg, dt); });
    }
    release(dg);
    release(dt);
    release(dc);
  }

  struct Plan {
    GemmTile* tiles = nullptr;
    GemmProb* probs = nullptr;
    GemmSeg* segs = nullptr;
    int ntiles = 0;
    bool live = false;
  };

  int gemm_plan(const std::vector<GemmProb>& p, const std::vector<GemmSeg>& s) override {
    Plan pl;
    std::vector<GemmTile> tiles;
    for (size_t i = 0; i < p.size(); ++i)
      for (int m0 = 0; m0 < p[i].M; m0 += TM)
        for (int n0 = 0; n0 < p[i].N; n0 += TN) tiles.push_back(GemmTile{int(i), m0, n0, 0});
    pl.ntiles = int(tiles.size());
    pl.tiles = upload(tiles);
    pl.probs = upload(p);
    pl.segs = upload(s);
    pl.live = true;
    for (size_t i = 0; i < plans_.size(); ++i)
      if (!plans_[i].live) {
        plans_[i] = pl;
        return int(i);
      }
    plans_.push_back(pl);
    return int(plans_.size() - 1);
  }
  void gemm_run(int id) override {
    Plan& pl = plans_.at(id);
    if (!pl.ntiles) return;
    launch(PROF_GEMM, [&] { gemm_f64_kernel<<<pl.ntiles, 256, 0, st_>>>(pl.tiles, pl.probs, pl.segs); });
  }
  void free_plan_mem(Plan& p) {
    if (!p.live) return;
    cudaFreeAsync(p.tiles, st_);
    cudaFreeAsync(p.probs, st_);
    cudaFreeAsync(p.segs, st_);
    p.live = false;
  }
  void plan_free(int id) override { free_plan_mem(plans_.at(id)); }
  void gemm(const std::vector<GemmProb>& p, const std::vector<GemmSeg>& s) override {
    if (p.empty()) return;
    int id = gemm_plan(p, s);
    gemm_run(id);
    plan_free(id);
  }
  void orbital_gradient(int L, const double* t, const double* v, const double* g1, const double* g2,
                        double* grad) override {
    double* F = static_cast<double*>(alloc(sizeof(double) * size_t(L) * L));
    launch(PROF_VEC, [&] { fock_kernel<<<L * L, 128, 0, st_>>>(L, t, v, g1, g2, F); });
    launch(PROF_VEC, [&] { orbital_grad_kernel<<<(L * L + 127) / 128, 128, 0, st_>>>(L, F, grad); });
    release(F);
  }
  void dots(const std::vector<DotTask>& t, double* out) override {
    if (t.empty()) return;
    DotTask* d = upload(t);
    const unsigned nb = unsigned(std::min<size_t>(t.size(), size_t(nsm_) * 16));
    launch(PROF_VEC, [&] { dot_tasks_kernel<<<nb, 128, 0, st_>>>(d, int(t.size()), out); });
    release(d);
  }
  void diag(const std::vector<DiagTask>& t) override {
    if (t.empty()) return;
    DiagTask* d = upload(t);
    launch(PROF_VEC, [&] { diag_kernel<<<std::min<size_t>(t.size(), 65535), 128, 0, st_>>>(d, int(t.size())); });
    release(d);
  }

  // ---- split-BF16 tensor-core path
  struct MixPlanD {
    MixTile* tiles = nullptr;
    MixProb* probs = nullptr;
    MixSeg* segs = nullptr;
    int64_t* bcol = nullptr;
    int64_t* ccol = nullptr;
    float* acol = nullptr;
    int* next_tile = nullptr;
    int ntiles = 0;
    int width = MIX_TN;
    int cls = PROF_MIXED;
    bool live = false;
    MixPlanHost host;
  };
  struct SplitPlanD {
    SplitTask* t = nullptr;
    int n = 0;
    bool live = false;
  };
  std::vector<MixPlanD> mplans_;
  std::vector<SplitPlanD> splans_;
  int* err_ = nullptr;

  int mix_plan(const std::vector<MixProb>& p, const std::vector<MixSeg>& s) override {
    return mix_plan_g(p, s, {}, {}, {});
  }
  int mix_plan_g(const std::vector<MixProb>& p, const std::vector<MixSeg>& s, const std::vector<int64_t>& bcol,
                 const std::vector<int64_t>& ccol, const std::vector<float>& acol) override {
    return mix_plan_ordered(p, s, bcol, ccol, acol, 0, MIX_TN);
  }
  int mix_plan_ordered(const std::vector<MixProb>& p, const std::vector<MixSeg>& s, const std::vector<int64_t>& bcol,
                       const std::vector<int64_t>& ccol, const std::vector<float>& acol, int order,
                       int width) override {
    if (order < 0 || order > 2) throw std::runtime_error("mix_plan: unknown tile order");
    if (!mix_width_ok(width)) throw std::runtime_error("mix_plan: tile width must be 32, 64 or 128");
    for (const MixSeg& g : s) {
      // blocked split matrices are built of 128-byte core-matrix pairs: every
      // bulk copy source is 16-byte aligned when the matrix base is
      if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(g.B) & 15) || g.K <= 0)
        throw std::runtime_error("mix_plan: operand not 16-byte aligned");
    }
    for (const MixProb& q : p) {
      if (q.mode < 0 || q.mode > 3 || q.mode == 1 || q.M <= 0 || q.N < 0 || q.s0 < 0 || q.s1 > int(s.size()) ||
          q.s0 > q.s1)
        throw std::runtime_error("mix_plan: bad problem");
      if (q.mode >= 2 && ((q.ldc & 31) || (q.N & 31) || q.N > q.ldc))
        throw std::runtime_error("mix_plan: bad split-matrix output");
      if (q.mode == 2 && (q.row0 < 0 || q.row0 + q.M > q.crows || (q.crows & 7)))
        throw std::runtime_error("mix_plan: bad dense-row problem");
      if (q.mode == 3 && ((q.cm0 & 7) || (q.M & 7) || q.cm0 < 0 || q.cm0 + q.M > int64_t(ccol.size()) ||
                          q.cm0 + q.M > int64_t(acol.size()) || (q.cm0 + q.M) / 4 > int64_t(bcol.size())))
        throw std::runtime_error("mix_plan: bad gathered problem");
      for (int k = q.s0; k < q.s1; ++k)
        if (s[k].A == nullptr || s[k].B == nullptr) throw std::runtime_error("mix_plan: bad segment");
    }
    std::vector<MixTile> tiles;
    std::vector<int64_t> work;
    for (size_t i = 0; i < p.size(); ++i) {
      int64_t w = 1;
      for (int q = p[i].s0; q < p[i].s1; ++q) w += (s[q].K + 31) / 32;
      for (int m0 = 0; m0 < p[i].M; m0 += MIX_TM)
        for (int n0 = 0; n0 < p[i].N; n0 += width) {
          tiles.push_back(MixTile{int(i), m0, n0, int(w - 1)});
          work.push_back(w);
        }
    }
    {
      // persistent CTAs take tiles in strides: longest first balances the load;
      // orders 1 and 2 keep each problem's tiles together (operand slabs shared
      // by the tiles of one output block are then read at about the same time)
      std::vector<size_t> ord(tiles.size());
      for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
      if (order == 0) {
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
      } else if (order == 2) {
        std::vector<int64_t> pw(p.size(), 0);
        for (size_t i = 0; i < tiles.size(); ++i) pw[tiles[i].prob] += work[i];
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
          const int pa = tiles[a].prob, pb = tiles[b].prob;
          return pa != pb && (pw[pa] != pw[pb] ? pw[pa] > pw[pb] : pa < pb);
        });
      }
      std::vector<MixTile> t2;
      t2.reserve(tiles.size());
      for (size_t i : ord) t2.push_back(tiles[i]);
      tiles.swap(t2);
    }
    MixPlanD pl;
    pl.ntiles = int(tiles.size());
    pl.width = width;
    pl.tiles = upload(tiles);
    pl.probs = upload(p);
    pl.segs = upload(s);
    pl.bcol = upload(bcol);
    pl.ccol = upload(ccol);
    pl.acol = upload(acol);
    pl.next_tile = static_cast<int*>(alloc(sizeof(int)));
    pl.live = true;
    pl.cls = (!p.empty() && p[0].mode != 0) ? PROF_MIXED1 : PROF_MIXED;
    pl.host = MixPlanHost{p, s, bcol, ccol, acol};
    for (size_t i = 0; i < mplans_.size(); ++i)
      if (!mplans_[i].live) {
        mplans_[i] = pl;
        return int(i);
      }
    mplans_.push_back(pl);
    return int(mplans_.size() - 1);
  }
  void mix_run(int id) override {
    MixPlanD& pl = mplans_.at(id);
    if (!pl.ntiles) return;
    launch(pl.cls, [&] {
      // tiles handed out through the counter where they are long (the K-concatenated
      // products of stage 2); in fixed strides where they are short (stage 1)
      int* nt = pl.cls == PROF_MIXED ? pl.next_tile : nullptr;
      launch_mixed_gemm(pl.tiles, pl.ntiles, pl.probs, pl.segs, pl.bcol, pl.ccol, pl.acol, err_, nt, pl.width, nsm_,
                        st_);
    });
  }
  void mix_plan_free(int id) override { mix_free(id); }
  const MixPlanHost& mix_plan_host(int id) const override { return mplans_.at(id).host; }
  float mix_time(int id, int reps) override {
    mix_run(id);
    cudaEvent_t a = ev(), b = ev();
    CK(cudaEventRecord(a, st_));
    for (int r = 0; r < reps; ++r) mix_run(id);
    CK(cudaEventRecord(b, st_));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    pool_.push_back(a);
    pool_.push_back(b);
    return ms / float(std::max(1, reps));
  }
  void* stream() const override { return st_; }
  bool profiling() const override { return prof_; }
  void split_plan_free(int id) override {
    SplitPlanD& pl = splans_.at(id);
    if (!pl.live) return;
    cudaFreeAsync(pl.t, st_);
    pl.live = false;
  }
  void mix_free(int id) {
    MixPlanD& pl = mplans_.at(id);
    if (!pl.live) return;
    cudaFreeAsync(pl.tiles, st_);
    cudaFreeAsync(pl.probs, st_);
    cudaFreeAsync(pl.segs, st_);
    cudaFreeAsync(pl.bcol, st_);
    cudaFreeAsync(pl.ccol, st_);
    cudaFreeAsync(pl.acol, st_);
    cudaFreeAsync(pl.next_tile, st_);
    pl.host = MixPlanHost{};
    pl.live = false;
  }
  int split_plan(const std::vector<SplitTask>& t) override {
    SplitPlanD pl;
    pl.n = int(t.size());
    pl.t = upload(t);
    pl.live = true;
    for (size_t i = 0; i < splans_.size(); ++i)
      if (!splans_[i].live) {
        splans_[i] = pl;
        return int(i);
      }
    splans_.push_back(pl);
    return int(splans_.size() - 1);
  }
  void split_run(int id) override {
    SplitPlanD& pl = splans_.at(id);
    if (!pl.n) return;
    launch(PROF_SPLIT, [&] { launch_split(pl.t, pl.n, st_); });
  }
  void df_to_f64(const float* hi, const float* lo, double* out, int64_t n) override {
    launch(PROF_SPLIT, [&] { launch_df_to_f64(hi, lo, out, n, grid_for(n), st_); });
  }
  void reduce_parts(const float* part, int nparts, int64_t n, float* hi, float* lo, int accumulate) override {
    launch(PROF_SPLIT, [&] { launch_reduce_parts(part, nparts, n, hi, lo, accumulate, grid_for(n), st_); });
  }
  int graph_capture(const std::function<void()>& f) override {
    if (st_ == nullptr || prof_) return -1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st_, &cs));
    if (cs != cudaStreamCaptureStatusNone) return -1;   // the caller is capturing already
    CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
    try {
      f();
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(st_, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamEndCapture(st_, &g));
    cudaGraphExec_t ge = nullptr;
    const cudaError_t rc = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(rc);
    for (size_t i = 0; i < graphs_.size(); ++i)
      if (!graphs_[i]) {
        graphs_[i] = ge;
        return int(i);
      }
    graphs_.push_back(ge);
    return int(graphs_.size() - 1);
  }
  void graph_run(int id) override { CK(cudaGraphLaunch(graphs_.at(id), st_)); }
  void graph_free(int id) override {
    if (id >= 0 && id < int(graphs_.size()) && graphs_[id]) {
      cudaGraphExecDestroy(graphs_[id]);
      graphs_[id] = nullptr;
    }
  }
  int device_error() override {
    int h = 0;
    CK(cudaMemcpyAsync(&h, err_, sizeof(int), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    return h;
  }

  int grid_for(int64_t n) const { return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, int64_t(nsm_) * 8))); }

  void mdot(const double* V, int64_t ldv, int m, const double* X, int64_t ldx, int k, int64_t n, double* out,
            int ldo) override {
    if (k > 4) throw std::runtime_error("mdot: at most 4 right-hand vectors");
    for (int i0 = 0; i0 < m; i0 += MDOT_MAX) {
      const int mm = std::min(MDOT_MAX, m - i0);
      const int nb = int(std::max<int64_t>(1, std::min<int64_t>((n + 4095) / 4096, 1024 / std::max(1, k))));
      launch(PROF_VEC, [&] { mdot_partial<<<dim3(nb, k), 256, 0, st_>>>(V + i0 * ldv, ldv, mm, X, ldx, n, part_); });
      launch(PROF_VEC, [&] { mdot_final<<<(mm * k + 127) / 128, 128, 0, st_>>>(part_, nb, mm, k, out + i0 * ldo, ldo); });
    }
  }
  void lincomb(const double* V, int64_t ldv, int m, const double* C, int ldc, int k, int64_t n, double* Y,
               int64_t ldy, double alpha, double beta) override {
    launch(PROF_VEC, [&] { lincomb_kernel<<<grid_for(n), 256, 0, st_>>>(V, ldv, m, C, ldc, k, n, Y, ldy, alpha, beta); });
  }
  void axpy_dev(const double* x, double* y, int64_t n, const double* s, double alpha) override {
    launch(PROF_VEC, [&] { axpy_dev_kernel<<<grid_for(n), 256, 0, st_>>>(x, y, n, s, alpha); });
  }
  void precond(const double* r, const double* d, const double* th, int64_t n, double* t, double fl) override {
    launch(PROF_VEC, [&] { precond_kernel<<<grid_for(n), 256, 0, st_>>>(r, d, th, n, t, fl); });
  }
  void normalize(double* x, int64_t n, const double* nrm2) override {
    launch(PROF_VEC, [&] { normalize_kernel<<<grid_for(n), 256, 0, st_>>>(x, n, nrm2); });
  }
  void ritz(const double* H, int ldh, int m, double* theta, double* y) override {
    if (m > 40) throw std::runtime_error("ritz: subspace larger than 40");
    launch(PROF_EIG, [&] { ritz_kernel<<<1, 64, 0, st_>>>(H, ldh, m, theta, y); });
  }
  void syev(const std::vector<double*>& A, const std::vector<double*>& w, const std::vector<double*>& Z,
            const std::vector<int>& n) override {
    if (A.empty()) return;
    const int nj = int(A.size());
    // per matrix: d, e, tau, pb (4n), Zc, U (2 n^2) doubles; perm (n) ints; every
    // part 16-byte aligned
    auto up2 = [](int64_t x) { return (x + 1) & ~int64_t(1); };
    auto up4 = [](int64_t x) { return (x + 3) & ~int64_t(3); };
    std::vector<int64_t> doff(nj), ioff(nj);
    std::vector<int> pre_n(nj + 1, 0);
    int64_t dtot = 0, itot = 0;
    int maxn = 2;
    for (int j = 0; j < nj; ++j) {
      const int64_t m = n[j];
      if (m <= 0) throw std::runtime_error("syev: empty matrix");
      if (m > 32767) throw std::runtime_error("syev: matrix order above 32767");
      doff[j] = dtot;
      dtot += up2(4 * m) + 2 * up2(m * m);
      ioff[j] = itot;
      itot += up4(m);
      pre_n[j + 1] = pre_n[j] + int(m);
      maxn = std::max(maxn, int(m) + 2);
    }
    const size_t smem1 = sizeof(double) * (2 * size_t(maxn) + 40);
    if (smem1 > 227 * 1024) throw std::runtime_error("syev: matrix too large for the shared-memory workspace");
    double* dw = static_cast<double*>(alloc(sizeof(double) * size_t(dtot)));
    int* iw = static_cast<int*>(alloc(sizeof(int) * size_t(itot)));
    std::vector<SyevJob> jobs(nj);
    for (int j = 0; j < nj; ++j) {
      const int64_t m = n[j];
      SyevJob& jb = jobs[j];
      double* p = dw + doff[j];
      jb.A = A[j];
      jb.w = w[j];
      jb.Z = Z[j];
      jb.d = p;
      jb.e = p + m;
      jb.tau = p + 2 * m;
      jb.pb = p + 3 * m;
      p += up2(4 * m);
      jb.Zc = p;
      p += up2(m * m);
      jb.U = p;
      jb.perm = iw + ioff[j];
      jb.n = int(m);
      jb.pad = 0;
    }
    // 1. the reduction: a cluster of SYEV_CLUSTER CTAs for each matrix of order >= 256,
    // one CTA for each smaller one; 2. Q
    std::vector<int> small, big;
    for (int j = 0; j < nj; ++j) (n[j] >= 256 ? big : small).push_back(j);
    SyevJob* dj = upload(jobs);
    int* dpn = upload(pre_n);
    int* dsmall = upload(small);
    int* dbig = upload(big);
    if (smem1 > 48 * 1024) {
      CK(cudaFuncSetAttribute(syev_tridiag_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem1)));
      CK(cudaFuncSetAttribute(syev_tridiag_kernel<SYEV_CLUSTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(smem1)));
    }
    const int ncol = pre_n[nj];
    if (!small.empty())
      launch(PROF_EIG, [&] {
        syev_tridiag_kernel<1><<<unsigned(small.size()), SYEV_THREADS, smem1, st_>>>(dj, dsmall, maxn);
      });
    if (!big.empty())
      launch(PROF_EIG, [&] {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(big.size() * SYEV_CLUSTER));
        cfg.blockDim = dim3(SYEV_THREADS);
        cfg.dynamicSmemBytes = smem1;
        cfg.stream = st_;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = SYEV_CLUSTER;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, syev_tridiag_kernel<SYEV_CLUSTER>, static_cast<const SyevJob*>(dj),
                              static_cast<const int*>(dbig), maxn));
      });
    launch(PROF_EIG, [&] { syev_qform_kernel<<<unsigned((ncol + 7) / 8), 256, 0, st_>>>(dj, dpn, nj); });
    // 3. T = V diag(d) V^T by divide and conquer: the blocks are halved until they
    // have at most DC_LEAF rows; a merge runs once both halves are solved, so the
    // merges go level by level (by the height of their subtree) over all matrices
    std::vector<DcLeaf> leaves;
    std::vector<std::vector<DcMerge>> levels;
    for (int j = 0; j < nj; ++j) {
      const SyevJob& jb = jobs[j];
      std::function<int(int, int)> split = [&](int o, int sz) -> int {
        if (sz <= DC_LEAF) {
          leaves.push_back(DcLeaf{jb.d, jb.e, jb.A, jb.n, o, sz, 0});
          return 0;
        }
        const int s1 = sz / 2;
        const int h = std::max(split(o, s1), split(o + s1, sz - s1)) + 1;
        if (int(levels.size()) < h) levels.resize(size_t(h));
        DcMerge mg{};
        mg.d = jb.d;
        mg.e = jb.e;
        mg.Z = jb.A;
        mg.n = jb.n;
        mg.o = o;
        mg.s1 = s1;
        mg.s = sz;
        levels[size_t(h - 1)].push_back(mg);
        return h;
      };
      split(0, jb.n);
    }
    DcLeaf* dl = upload(leaves);
    launch(PROF_EIG, [&] { launch_dc_leaves(dl, int(leaves.size()), err_, st_); });
    std::vector<void*> scratch;
    for (auto& lv : levels) {
      // scratch per merge: doubles 8 s + 2 s^2 + 2, ints 5 s + 4 (16-byte aligned parts)
      int64_t nd = 0, ni = 0;
      for (const DcMerge& mg : lv) {
        nd += up2(8 * int64_t(mg.s) + 2) + 2 * up2(int64_t(mg.s) * mg.s);
        ni += up4(5 * int64_t(mg.s) + 4);
      }
      double* sd = static_cast<double*>(alloc(sizeof(double) * size_t(nd)));
      int* si = static_cast<int*>(alloc(sizeof(int) * size_t(ni)));
      scratch.push_back(sd);
      scratch.push_back(si);
      std::vector<int> ps(lv.size() + 1, 0), pt(lv.size() + 1, 0);
      int64_t od = 0, oi = 0;
      for (size_t i = 0; i < lv.size(); ++i) {
        DcMerge& mg = lv[i];
        const int64_t s = mg.s;
        double* p = sd + od;
        mg.ds = p;
        mg.zs = p + s;
        mg.dk = p + 2 * s;
        mg.zk = p + 3 * s;
        mg.tau = p + 4 * s;
        mg.zh = p + 5 * s;
        mg.gc = p + 6 * s;
        mg.gs = p + 7 * s;
        mg.rho = p + 8 * s;
        p += up2(8 * s + 2);
        mg.Qp = p;
        p += up2(s * s);
        mg.U = p;
        od += up2(8 * s + 2) + 2 * up2(s * s);
        int* q = si + oi;
        mg.perm = q;
        mg.ndp = q + s;
        mg.org = q + 2 * s;
        mg.gp = q + 3 * s;
        mg.cnt = q + 5 * s;
        oi += up4(5 * s + 4);
        const int nt = int((s + 63) / 64);
        ps[i + 1] = ps[i] + int(s);
        pt[i + 1] = pt[i] + nt * nt;
      }
      DcMerge* dm = upload(lv);
      int* dps = upload(ps);
      int* dpt = upload(pt);
      launch(PROF_EIG, [&] {
        launch_dc_merges(dm, int(lv.size()), dps, ps.back(), dpt, pt.back(), st_);
      });
      release(dm);
      release(dps);
      release(dpt);
    }
    // 4. W = Q V (column-major both: as row-major arrays W^T = V^T Q^T), into U
    {
      std::vector<GemmProb> P;
      std::vector<GemmSeg> S;
      for (const SyevJob& jb : jobs) {
        GemmProb q;
        q.C = jb.U;
        q.ldc = jb.n;
        q.M = jb.n;
        q.N = jb.n;
        q.alpha = 1.0;
        q.accumulate = 0;
        q.s0 = int(S.size());
        S.push_back(GemmSeg{jb.A, jb.Zc, jb.n, jb.n, jb.n, 0, 0});
        q.s1 = int(S.size());
        P.push_back(q);
      }
      gemm(P, S);
    }
    // 5. order
    launch(PROF_EIG, [&] { syev_sort_kernel<<<unsigned((ncol + 255) / 256), 256, 0, st_>>>(dj, dpn, nj); });
    launch(PROF_EIG, [&] { syev_perm_kernel<<<unsigned(ncol), 128, 0, st_>>>(dj, dpn, nj); });
    for (void* p : scratch) release(p);
    release(dl);
    release(dj);
    release(dpn);
    release(dsmall);
    release(dbig);
    release(dw);
    release(iw);
  }

 private:
  cudaStream_t st_;
  int prec_;
  int dev_ = 0, nsm_ = 148;
  int64_t n_alloc_ = 0;
  cudaMemPool_t mpool_ = nullptr;
  static constexpr size_t kStageMax = size_t(512) << 20;   // pinned staging ring: at most 512 MiB
  char* stage_ = nullptr;
  size_t stage_cap_ = 0, stage_head_ = 0;
  cudaEvent_t stage_ev_ = nullptr;
  std::vector<cudaGraphExec_t> graphs_;
  double* part_ = nullptr;
  std::vector<Plan> plans_;
};

Exec* make_cuda_exec(void* stream, int precision_mode) { return new CudaExec(stream, precision_mode); }

}  // namespace dmrg
