// Split-BF16 tensor-core path (tcgen05 / TMEM) shared by exec_cuda.cu and mixed.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../exec.h"

namespace dmrg {

struct MixTile {
  int prob, m0, n0;
  int nsteps;   // K stages of the tile (sum over its segments of ceil(K / 32))
};

// launch the grouped split-BF16 GEMM over `ntiles` tiles; err is a device int
// that receives a nonzero code when a bounded wait gives up; next_tile, when not
// null, is a device int through which the launch hands out tiles in list order
// (cleared by the launch; one per plan), else CTAs take tiles in fixed strides;
// tn is the tile width of the list (MMA N: 32, 64 or 128; tile columns start at
// multiples of tn)
void launch_mixed_gemm(const MixTile* tiles, int ntiles, const MixProb* probs, const MixSeg* segs,
                       const int64_t* bcol, const int64_t* ccol, const float* acol, int* err, int* next_tile,
                       int tn, int nsm, cudaStream_t st);
void launch_split(const SplitTask* t, int ntask, cudaStream_t st);
void launch_reduce_parts(const float* part, int nparts, int64_t n, float* hi, float* lo, int accumulate, int grid,
                         cudaStream_t st);
void launch_df_to_f64(const float* hi, const float* lo, double* out, int64_t n, int grid, cudaStream_t st);

constexpr int MIX_TM = 128;   // rows per tile (MMA M)
constexpr int MIX_TN = 128;   // max columns per tile (MMA N, rounded to 16 per tile)
// tile widths a plan may use (the batched form's autotuner chooses among them)
inline bool mix_width_ok(int w) { return w == 32 || w == 64 || w == MIX_TN; }

}  // namespace dmrg
