// Divide-and-conquer eigensolver of symmetric tridiagonal matrices (the
// eigenvector step of the density-matrix diagonalisation of the truncation).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace dmrg {

// One leaf: rows [o, o + s) of a job's tridiagonal matrix (s <= DC_LEAF), solved
// by implicit QL on one warp; the tear couplings at both ends are taken off the
// diagonal first.
struct DcLeaf {
  double* d;   // job diagonal (n): on exit d[o..o+s) = the leaf's eigenvalues
  const double* e;   // job off-diagonal (n): e[i] couples i and i + 1
  double* Z;   // job eigenvectors (n x n, column-major): diagonal block [o, o+s) written
  int n, o, s, pad;
};

// One merge: the two solved blocks [o, o + s1) and [o + s1, o + s) of a job and the
// coupling e[o + s1 - 1] between them give the eigenpairs of the block [o, o + s).
struct DcMerge {
  double* d;
  const double* e;
  double* Z;
  int n, o, s1, s;
  // scratch (device, owned by the caller): doubles 8 s + 2 + 2 s^2, ints 5 s + 4
  double* ds;   // s: sorted diagonal (after the deflation rotations)
  double* zs;   // s: sorted z (after the deflation rotations)
  double* dk;   // s: the k non-deflated ds, ascending
  double* zk;   // s: their z
  double* tau;  // s: secular roots as offsets from their origin pole
  double* zh;   // s: z recomputed from the roots (Gu-Eisenstat)
  double* gc;   // s: deflation rotations (cosine, sine); first z and d of the two blocks
  double* gs;
  double* Qp;   // s x s column-major: the two blocks' eigenvectors, sorted and rotated
  double* U;    // k x k column-major: eigenvectors of diag(dk) + rho zk zk^T
  int* perm;    // s: sorted position -> column of the two blocks
  int* ndp;     // s: j-th non-deflated sorted position
  int* org;     // s: origin pole of root j
  int* gp;      // 2 s: slot 2 q the q-th deflation rotation's pair p | i << 16, slot 2 i + 1
                //      pole i's flag (-1 deflated, 0 kept)
  int* cnt;     // 4: k, number of deflation rotations
  double* rho;  // 1: the rank-one weight rho ||z||^2
};

constexpr int DC_LEAF = 32;

void launch_dc_leaves(const DcLeaf* leaves, int nleaves, int* err, cudaStream_t st);
// pre_s: prefix sums of the merges' s (device, nmerge + 1 entries); total = pre_s[nmerge];
// tiles: prefix sums of ceil(s/32)^2 (device), ttotal its last entry
void launch_dc_merges(const DcMerge* m, int nmerge, const int* pre_s, int total, const int* pre_t, int ttotal,
                      cudaStream_t st);

}  // namespace dmrg
