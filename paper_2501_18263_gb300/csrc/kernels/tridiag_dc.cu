// Divide-and-conquer symmetric tridiagonal eigensolver (Cuppen, "A divide and
// conquer method for the symmetric tridiagonal eigenproblem", Numer. Math. 36
// (1981); eigenvectors by Gu and Eisenstat, "A divide-and-conquer algorithm for the
// symmetric tridiagonal eigenproblem", SIAM J. Matrix Anal. Appl. 16 (1995)).
//
// T is torn at every block boundary: with beta = T[b-1, b] and rho = |beta|,
// T = diag(T_1, T_2) + rho v v^T, v = e_{b-1} + sign(beta) e_b, where T_1, T_2 have
// their corner diagonal entries lowered by rho.  The leaves (at most 32 rows) are
// solved by implicit QL on one warp each.  A merge of two solved blocks with
// eigenpairs (D_i, Q_i) is the eigenproblem of D + rho z z^T, z = Q^T v (the last
// row of Q_1, sign(beta) times the first row of Q_2):
//  1. z normalised (rho takes ||z||^2), D sorted;
//  2. deflation: a component with rho |z_i| <= tol keeps (d_i, column i); of two
//     close poles a plane rotation zeroes the earlier z and keeps it when the
//     coupling it leaves, |(d_i - d_p) c s|, is below tol
//     (tol = 8 eps max(max |d|, rho));
//  3. the k roots of 1 + rho sum_i z_i^2 / (d_i - lambda) = 0, root j in
//     (d_j, d_{j+1}) (the last in (d_k, d_k + rho sum z^2)), each as an offset tau
//     from its nearer pole, by bisection on the bit patterns of tau (one warp per
//     root, the sum over the lanes);
//  4. z recomputed from the roots, zh_i^2 = prod_j (lambda_j - d_i) /
//     (rho prod_{l != i} (d_l - d_i)), so that the eigenvectors u_j = zh / (d - lambda_j)
//     are orthogonal to working accuracy;
//  5. the new eigenvectors Q [u_j] by an FP64 GEMM per merge.
// Every difference d_i - lambda_j is formed as (d_i - d_org(j)) - tau_j.
#include "tridiag_dc.h"

#include <cstdint>

namespace dmrg {
namespace {

__device__ __forceinline__ double dc_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int dc_find(const int* pre, int nj, int x) {
  int lo = 0, hi = nj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---- leaves: one warp each, lane r holds row r of the leaf's eigenvectors in
// shared memory; lane 0 runs the QL recurrences of one iteration and records its
// rotations, then every lane applies them to its row.  More than 60 iterations for
// one eigenvalue: *err = 9.
constexpr int DC_LEAF_WARPS = 4;

__global__ void __launch_bounds__(32 * DC_LEAF_WARPS) dc_leaf_kernel(const DcLeaf* __restrict__ leaves, int nl,
                                                                    int* err) {
  __shared__ double zsm[DC_LEAF_WARPS][DC_LEAF][DC_LEAF + 1];
  __shared__ double dsm[DC_LEAF_WARPS][DC_LEAF], esm[DC_LEAF_WARPS][DC_LEAF];
  __shared__ double rc[DC_LEAF_WARPS][DC_LEAF], rs[DC_LEAF_WARPS][DC_LEAF];
  __shared__ int ctl[DC_LEAF_WARPS][2];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int li = blockIdx.x * DC_LEAF_WARPS + w;
  if (li >= nl) return;
  const DcLeaf lf = leaves[li];
  const int s = lf.s, o = lf.o, n = lf.n;
  double (*Zl)[DC_LEAF + 1] = zsm[w];
  double* dd = dsm[w];
  double* ee = esm[w];
  if (lane < s) {
    double dv = lf.d[o + lane];
    if (lane == 0 && o > 0) dv -= fabs(lf.e[o - 1]);             // tear above the leaf
    if (lane == s - 1 && o + s < n) dv -= fabs(lf.e[o + s - 1]);  // tear below it
    dd[lane] = dv;
    ee[lane] = lane < s - 1 ? lf.e[o + lane] : 0.0;
    for (int c = 0; c < s; ++c) Zl[lane][c] = (c == lane) ? 1.0 : 0.0;
  }
  __syncwarp();
  const double eps = 2.220446049250313e-16;
  int l = 0, iter = 0;
  double tnorm = 0.0;
  if (lane == 0)
    for (int i = 0; i < s; ++i) tnorm = fmax(tnorm, fabs(dd[i]) + fabs(ee[i]) + (i ? fabs(ee[i - 1]) : 0.0));
  for (;;) {
    if (lane == 0) {
      int nrot = -1, first = 0;
      while (l < s) {
        int mm = l;
        for (; mm < s - 1; ++mm)
          if (fabs(ee[mm]) <= eps * (fabs(dd[mm]) + fabs(dd[mm + 1])) || fabs(ee[mm]) <= eps * tnorm) break;
        if (mm == l) {
          ++l;
          iter = 0;
          continue;
        }
        if (++iter > 60) {
          atomicExch(err, 9);
          l = s;
          break;
        }
        double g = (dd[l + 1] - dd[l]) / (2.0 * ee[l]);
        double r = hypot(g, 1.0);
        g = dd[mm] - dd[l] + ee[l] / (g + (g >= 0.0 ? r : -r));
        double sn = 1.0, c = 1.0, p = 0.0;
        bool split = false;
        nrot = 0;
        first = mm - 1;
        for (int i = mm - 1; i >= l; --i) {
          const double f = sn * ee[i], b = c * ee[i];
          r = hypot(f, g);
          ee[i + 1] = r;
          if (r == 0.0) {
            dd[i + 1] -= p;
            ee[mm] = 0.0;
            split = true;
            break;
          }
          sn = f / r;
          c = g / r;
          g = dd[i + 1] - p;
          r = (dd[i] - g) * sn + 2.0 * c * b;
          p = sn * r;
          dd[i + 1] = g + p;
          g = c * r - b;
          rc[w][nrot] = c;
          rs[w][nrot] = sn;
          ++nrot;
        }
        if (!split) {
          dd[l] -= p;
          ee[l] = g;
          ee[mm] = 0.0;
        }
        break;
      }
      ctl[w][0] = (l < s) ? nrot : -1;
      ctl[w][1] = first;
    }
    __syncwarp();
    const int nrot = ctl[w][0], first = ctl[w][1];
    if (nrot < 0) break;
    if (lane < s) {
      // rotation q mixes columns i = first - q and i + 1 of row `lane`
      double zi1 = Zl[lane][first + 1];
      for (int q = 0; q < nrot; ++q) {
        const int i = first - q;
        const double c = rc[w][q], sn = rs[w][q];
        const double zi = Zl[lane][i];
        Zl[lane][i + 1] = sn * zi + c * zi1;
        zi1 = c * zi - sn * zi1;
      }
      if (nrot > 0) Zl[lane][first - nrot + 1] = zi1;
    }
    __syncwarp();
  }
  if (lane < s) {
    lf.d[o + lane] = dd[lane];
    // column c of the leaf is column o + c of Z, rows o .. o + s - 1
    for (int c = 0; c < s; ++c) lf.Z[int64_t(o + c) * n + o + lane] = Zl[lane][c];
  }
}

// ---- merge step 1-2: one CTA per merge.  z from the two blocks' boundary rows,
// normalised; poles sorted (rank of each); deflation on one thread (sequential
// over the sorted poles, as the pairing with the previous kept pole requires).
constexpr int DC_PREP_THREADS = 256;

__device__ double dc_block_sum(double v, double* red) {
  v = dc_warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = lane < int(blockDim.x >> 5) ? red[lane] : 0.0;
    x = dc_warp_sum(x);
    if (lane == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}

__global__ void __launch_bounds__(DC_PREP_THREADS) dc_prep_kernel(const DcMerge* __restrict__ ms) {
  __shared__ double red[34];
  const DcMerge m = ms[blockIdx.x];
  const int s = m.s, s1 = m.s1, o = m.o, n = m.n;
  const double beta = m.e[o + s1 - 1];
  const double sg = beta >= 0.0 ? 1.0 : -1.0;
  // z_i (column i of the two blocks) into gc temporarily, d into gs
  double part = 0.0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const double zi = i < s1 ? m.Z[int64_t(o + i) * n + (o + s1 - 1)] : sg * m.Z[int64_t(o + i) * n + (o + s1)];
    m.gc[i] = zi;
    m.gs[i] = m.d[o + i];
    part += zi * zi;
  }
  const double nz2 = dc_block_sum(part, red);
  const double inv = nz2 > 0.0 ? 1.0 / sqrt(nz2) : 0.0;
  // rank sort (ties by index)
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const double di = m.gs[i];
    int r = 0;
    for (int j = 0; j < s; ++j) {
      const double dj = m.gs[j];
      r += (dj < di) || (dj == di && j < i);
    }
    m.ds[r] = di;
    m.zs[r] = m.gc[i] * inv;
    m.perm[r] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double rho = fabs(beta) * nz2;
    double dmax = 0.0;
    for (int i = 0; i < s; ++i) dmax = fmax(dmax, fabs(m.ds[i]));
    const double tol = 8.0 * 2.220446049250313e-16 * fmax(dmax, rho);
    int ng = 0, k = 0, p = -1;
    for (int i = 0; i < s; ++i) {
      if (rho * fabs(m.zs[i]) <= tol) {   // deflated: (ds_i, column i) stays an eigenpair
        m.gp[2 * i + 1] = -1;             // mark (the pair slots double as flags below)
        continue;
      }
      m.gp[2 * i + 1] = 0;
      if (p >= 0) {
        const double t = hypot(m.zs[p], m.zs[i]);
        const double c = m.zs[i] / t, sn = -m.zs[p] / t;
        if (fabs((m.ds[i] - m.ds[p]) * c * sn) <= tol) {
          // rotate columns p, i so that z_p = 0; pole p deflates
          const double dp = m.ds[p] * c * c + m.ds[i] * sn * sn;
          const double di = m.ds[p] * sn * sn + m.ds[i] * c * c;
          m.ds[p] = dp;
          m.ds[i] = di;
          m.zs[p] = 0.0;
          m.zs[i] = t;
          m.gp[2 * p + 1] = -1;
          m.gc[ng] = c;
          m.gs[ng] = sn;
          m.gp[2 * ng] = p | (i << 16);
          ++ng;
        }
      }
      p = i;
    }
    for (int i = 0; i < s; ++i)
      if (m.gp[2 * i + 1] == 0) {
        m.ndp[k] = i;
        m.dk[k] = m.ds[i];
        m.zk[k] = m.zs[i];
        ++k;
      }
    m.cnt[0] = k;
    m.cnt[1] = ng;
    m.rho[0] = rho;
  }
}

// ---- merge step 3: one warp per root (pre_s: prefix sums of the merges' s; root
// slots past k exit).  f(lambda) rises from -inf to +inf between poles; the root is
// bracketed on the half of (d_j, d_{j+1}) where it lies and tau is bisected over
// its bit patterns (non-negative doubles order like their bit patterns), at most 63
// steps to adjacent doubles.
__global__ void __launch_bounds__(256) dc_secular_kernel(const DcMerge* __restrict__ ms, int nm,
                                                         const int* __restrict__ pre_s) {
  const int gw = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (gw >= pre_s[nm]) return;
  const int mi = dc_find(pre_s, nm, gw);
  const DcMerge m = ms[mi];
  const int j = gw - pre_s[mi];
  const int k = m.cnt[0];
  if (j >= k) return;
  const double rho = m.rho[0];
  const double* dk = m.dk;
  const double* zk = m.zk;
  const double a = dk[j];
  double b;
  if (j + 1 < k) {
    b = dk[j + 1];
  } else {
    double z2 = 0.0;
    for (int i = lane; i < k; i += 32) z2 += zk[i] * zk[i];
    b = a + rho * dc_warp_sum(z2);
  }
  const double mid = 0.5 * (a + b);
  double fm = 0.0;
  for (int i = lane; i < k; i += 32) fm += zk[i] * zk[i] / (dk[i] - mid);
  fm = 1.0 + rho * dc_warp_sum(fm);
  int og;
  double sgn, hi;
  if (j + 1 == k || fm > 0.0) {
    og = j;
    sgn = 1.0;
    hi = (j + 1 < k) ? mid - a : b - a;
  } else {
    og = j + 1;
    sgn = -1.0;
    hi = b - mid;
  }
  const double dorg = dk[og];
  long long ilo = 0, ihi = __double_as_longlong(hi);
  while (ihi - ilo > 1) {
    const long long im = ilo + ((ihi - ilo) >> 1);
    const double t = sgn * __longlong_as_double(im);
    double f = 0.0;
    for (int i = lane; i < k; i += 32) f += zk[i] * zk[i] / ((dk[i] - dorg) - t);
    f = 1.0 + rho * dc_warp_sum(f);
    if ((f < 0.0) == (sgn > 0.0)) ilo = im;
    else ihi = im;
  }
  if (lane == 0) {
    m.org[j] = og;
    m.tau[j] = sgn * __longlong_as_double(ihi);
  }
}

// ---- merge step 4a: zh_i from the roots, one thread per (merge, i)
__global__ void __launch_bounds__(256) dc_zhat_kernel(const DcMerge* __restrict__ ms, int nm,
                                                      const int* __restrict__ pre_s) {
  const int g = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= pre_s[nm]) return;
  const int mi = dc_find(pre_s, nm, g);
  const DcMerge m = ms[mi];
  const int i = g - pre_s[mi];
  const int k = m.cnt[0];
  if (i >= k) return;
  const double rho = m.rho[0];
  const double di = m.dk[i];
  // lambda_j - d_i = tau_j - (d_i - d_org(j)); pair every factor with a pole gap
  double prod = (m.tau[i] - (di - m.dk[m.org[i]])) / rho;
  for (int j = 0; j < k; ++j) {
    if (j == i) continue;
    prod *= (m.tau[j] - (di - m.dk[m.org[j]])) / (m.dk[j] - di);
  }
  m.zh[i] = copysign(sqrt(fmax(prod, 0.0)), m.zk[i]);
}

// ---- merge step 4b: column j of U (k x k, column-major), normalised; one thread
// per (merge, j)
__global__ void __launch_bounds__(256) dc_ucol_kernel(const DcMerge* __restrict__ ms, int nm,
                                                      const int* __restrict__ pre_s) {
  const int g = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= pre_s[nm]) return;
  const int mi = dc_find(pre_s, nm, g);
  const DcMerge m = ms[mi];
  const int j = g - pre_s[mi];
  const int k = m.cnt[0];
  if (j >= k) return;
  const double dorg = m.dk[m.org[j]], tj = m.tau[j];
  double* u = m.U + int64_t(j) * k;
  double nrm = 0.0;
  for (int i = 0; i < k; ++i) {
    const double v = m.zh[i] / ((m.dk[i] - dorg) - tj);
    u[i] = v;
    nrm += v * v;
  }
  const double inv = 1.0 / sqrt(nrm);
  for (int i = 0; i < k; ++i) u[i] *= inv;
}

// ---- merge step 5a: Qp = the two blocks' eigenvectors (block diagonal), columns
// in sorted order, then the deflation rotations; one thread per (merge, row)
__global__ void __launch_bounds__(256) dc_qp_kernel(const DcMerge* __restrict__ ms, int nm,
                                                    const int* __restrict__ pre_s) {
  const int g = int(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= pre_s[nm]) return;
  const int mi = dc_find(pre_s, nm, g);
  const DcMerge m = ms[mi];
  const int r = g - pre_s[mi];
  const int s = m.s, s1 = m.s1, o = m.o, n = m.n;
  const bool top = r < s1;
  for (int c = 0; c < s; ++c) {
    const int src = m.perm[c];
    m.Qp[int64_t(c) * s + r] = ((src < s1) == top) ? m.Z[int64_t(o + src) * n + o + r] : 0.0;
  }
  const int ng = m.cnt[1];
  for (int q = 0; q < ng; ++q) {
    const int pr = m.gp[2 * q], p = pr & 0xffff, i = pr >> 16;
    const double c = m.gc[q], sn = m.gs[q];
    double* qp = m.Qp + int64_t(p) * s + r;
    double* qi = m.Qp + int64_t(i) * s + r;
    const double a = *qp, b = *qi;
    *qp = c * a + sn * b;
    *qi = -sn * a + c * b;
  }
}

// ---- merge step 5b: the new eigenvectors of the non-deflated poles,
// Z[:, o + ndp[j]] = Qp[:, ndp] U[:, j] (s x k times k x k), 64 x 64 tiles
// (pre_t: prefix sums of the merges' ceil(s/64)^2 tiles; tiles past k exit), and
// the new eigenvalues d_org(j) + tau_j
constexpr int DG_T = 64, DG_K = 16;

__global__ void __launch_bounds__(256) dc_gemm_kernel(const DcMerge* __restrict__ ms, int nm,
                                                      const int* __restrict__ pre_t) {
  __shared__ double As[DG_K][DG_T + 1];
  __shared__ double Bs[DG_K][DG_T + 1];
  const int mi = dc_find(pre_t, nm, int(blockIdx.x));
  const DcMerge m = ms[mi];
  const int s = m.s, k = m.cnt[0], o = m.o, n = m.n;
  const int ntc = (s + DG_T - 1) / DG_T;
  const int t = int(blockIdx.x) - pre_t[mi];
  const int r0 = (t / ntc) * DG_T, c0 = (t % ntc) * DG_T;
  if (c0 >= k) return;
  const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < k; k0 += DG_K) {
    for (int e = threadIdx.x; e < DG_T * DG_K; e += blockDim.x) {
      const int rr = e % DG_T, kk = e / DG_T;
      const int r = r0 + rr, kq = k0 + kk;
      As[kk][rr] = (r < s && kq < k) ? m.Qp[int64_t(m.ndp[kq]) * s + r] : 0.0;
    }
    for (int e = threadIdx.x; e < DG_T * DG_K; e += blockDim.x) {
      const int kk = e % DG_K, cc = e / DG_K;
      const int c = c0 + cc, kq = k0 + kk;
      Bs[kk][cc] = (c < k && kq < k) ? m.U[int64_t(c) * k + kq] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < DG_K; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + tc + 16 * j;
    if (c >= k) continue;
    double* zc = m.Z + int64_t(o + m.ndp[c]) * n + o;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + tr + 16 * i;
      if (r < s) zc[r] = acc[i][j];
    }
  }
}

// ---- merge step 5c: eigenvalues of the merged block; deflated columns copied
// from Qp.  One CTA per (merge, sorted position).
__global__ void __launch_bounds__(128) dc_finish_kernel(const DcMerge* __restrict__ ms, int nm,
                                                        const int* __restrict__ pre_s) {
  const int mi = dc_find(pre_s, nm, int(blockIdx.x));
  const DcMerge m = ms[mi];
  const int c = int(blockIdx.x) - pre_s[mi];
  const int s = m.s, o = m.o, n = m.n, k = m.cnt[0];
  if (m.gp[2 * c + 1] == -1) {   // deflated
    if (threadIdx.x == 0) m.d[o + c] = m.ds[c];
    const double* src = m.Qp + int64_t(c) * s;
    double* dst = m.Z + int64_t(o + c) * n + o;
    for (int r = threadIdx.x; r < s; r += blockDim.x) dst[r] = src[r];
  } else if (threadIdx.x == 0) {
    // c = ndp[j] for one j (ndp ascending): the root j
    int lo = 0, hi = k - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (m.ndp[mid] < c) lo = mid + 1;
      else hi = mid;
    }
    m.d[o + c] = m.dk[m.org[lo]] + m.tau[lo];
  }
}

}  // namespace

void launch_dc_leaves(const DcLeaf* leaves, int nleaves, int* err, cudaStream_t st) {
  if (nleaves <= 0) return;
  const unsigned g = unsigned((nleaves + DC_LEAF_WARPS - 1) / DC_LEAF_WARPS);
  dc_leaf_kernel<<<g, 32 * DC_LEAF_WARPS, 0, st>>>(leaves, nleaves, err);
}

void launch_dc_merges(const DcMerge* m, int nmerge, const int* pre_s, int total, const int* pre_t, int ttotal,
                      cudaStream_t st) {
  if (nmerge <= 0) return;
  dc_prep_kernel<<<unsigned(nmerge), DC_PREP_THREADS, 0, st>>>(m);
  dc_secular_kernel<<<unsigned((total + 7) / 8), 256, 0, st>>>(m, nmerge, pre_s);
  dc_zhat_kernel<<<unsigned((total + 255) / 256), 256, 0, st>>>(m, nmerge, pre_s);
  dc_ucol_kernel<<<unsigned((total + 255) / 256), 256, 0, st>>>(m, nmerge, pre_s);
  dc_qp_kernel<<<unsigned((total + 255) / 256), 256, 0, st>>>(m, nmerge, pre_s);
  dc_gemm_kernel<<<unsigned(ttotal), 256, 0, st>>>(m, nmerge, pre_t);
  dc_finish_kernel<<<unsigned(total), 128, 0, st>>>(m, nmerge, pre_s);
}

}  // namespace dmrg
