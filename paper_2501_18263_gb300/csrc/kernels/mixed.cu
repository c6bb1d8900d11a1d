// Split-BF16 grouped GEMM on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// Each operand x is carried as three BF16 planes with x ~ hi + mid + lo
// (residual below 2^-27 |x|).  A tile computes
//     acc0 = sum hi_A hi_B                                   (TMEM columns [0, 128))
//     acc1 = sum hi mid + mid hi + hi lo + mid mid + lo hi   (TMEM columns [128, 256))
// so that the rounding of the five small products happens in an accumulator
// 2^8 smaller than the result.  Every product of two BF16 values is exact in
// FP32, but the tensor core's FP32 accumulation loses about a third of an ulp
// per K = 16 step, so the accumulators only ever hold one chunk of K (CHUNK
// stages): after each chunk the drain warps fold them into a double-float
// running sum (hi + lo, TwoSum) held in registers.
//
// Every operand plane lives in HBM in the tensor core's core-matrix tiling (8
// rows x 16 bytes per core matrix, the K groups of an 8-row group contiguous), so
// the slice of one plane that a stage needs is one contiguous run of at most 512
// bytes per 8-row group, moved by cp.async.bulk straight into the canonical
// no-swizzle K-major shared-memory layout.  A ring of STAGES (three) stages is
// guarded by mbarriers (the full barriers count the copies' bytes); every wait is bounded
// and sets an error word instead of hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "mixed.h"

namespace dmrg {
namespace {

constexpr int BK = 32;                          // K elements per stage (one K slab)
constexpr int STAGES = 3;
constexpr int RG_BYTES = 3 * 8 * BK * 2;        // one 8-row group of a slab, three planes: 1536 B
constexpr int OPER_BYTES = 16 * RG_BYTES;       // a 128-row operand slab: 24 KiB
constexpr int STAGE_BYTES = 2 * OPER_BYTES;     // A and B
constexpr int BAR_BYTES = 256;
constexpr int DRAIN_THREADS = 512;              // 16 warps: 4 lane quarters x 4 column quarters
constexpr int DRAIN_COLS = 32;                  // accumulator columns per drain thread
constexpr int NTHREADS = 32 + 32 + DRAIN_THREADS;
constexpr int CHUNK = 8;                        // K stages per accumulator chunk (256 K)
constexpr long long WAIT_CYCLES = 3000000000LL; // about 1.5 s at 2 GHz (fits the 32-bit clock)
constexpr uint32_t TMEM_COLS = 512;

static_assert(MIX_TN == MIX_TM && MIX_TM == 128, "tiles are 128 x 128");

// control word of a ring stage, written by the producer beside the stage's data
struct StageInfo {
  int ksub;   // K = 16 MMA steps in the stage (1 or 2); 0: no more stages
  int last;   // last stage of its tile
  int nmma;   // MMA N of the tile
  int pad;
};
// per-tile record handed from the producer to the drain warps (double-buffered)
struct alignas(16) TileSlot {
  int64_t c[MIX_TM];   // mode 3: output-row table entries of the tile's rows
  float a[MIX_TM];     // mode 3: row scales
  float* Chi;
  float* Clo;
  uint16_t* Cp;
  int m0, n0, Nt, nch;
  int M, ldc, mode, pad0;
  int row0, crows;
  float alpha;
  int pad;
};
constexpr int SLOT_OFF = STAGES * STAGE_BYTES;
constexpr int INFO_OFF = SLOT_OFF + 2 * static_cast<int>(sizeof(TileSlot));
constexpr int BAR_OFF = INFO_OFF + STAGES * static_cast<int>(sizeof(StageInfo));
constexpr int SMEM_BYTES = BAR_OFF + BAR_BYTES;
static_assert(sizeof(TileSlot) % 16 == 0 && SMEM_BYTES <= 232448, "shared memory layout");

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: gives up after about WAIT_CYCLES SM cycles (32-bit clock, one
// wrap allowed) or when another role aborted, then raises the abort flag and
// records `code`.  Kept small in registers: the drain warps wait while holding
// their accumulator sums.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
  if (mbar_try(a, parity)) return true;
  const uint32_t t0 = static_cast<uint32_t>(clock());
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try(a, parity)) return true;
    if ((spin & 255u) == 0 &&
        (*abort_flag || static_cast<uint32_t>(clock()) - t0 > static_cast<uint32_t>(WAIT_CYCLES))) {
      if (!*abort_flag) {
        *abort_flag = 1;
        atomicExch(err, code);
      }
      return false;
    }
  }
}

// wait bounded by time alone (used on the way out, after an abort, for the
// kernel's own asynchronous copies and MMAs still in flight)
__device__ void mbar_wait_exit(uint32_t a, uint32_t parity, int* err) {
  const long long t0 = clock64();
  while (!mbar_try(a, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(err, 5);
      return;
    }
  }
}

// warp-level bounded wait: one lane polls the barrier, the other lanes wait at
// the __syncwarp (so that hundreds of threads do not spin on shared memory)
__device__ __forceinline__ bool mbar_wait_warp(uint32_t a, uint32_t parity, volatile int* abort_flag, int* err,
                                               int code) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(a, parity, abort_flag, err, code) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle,
// core matrices of 8 rows x 16 bytes; LBO = 128 B (next core matrix along K),
// SBO = 1536 B (next 8-row group along M/N: the three planes of a group are
// interleaved, plane q at +512 q)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((128u >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((static_cast<uint32_t>(RG_BYTES) >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;  // descriptor version of the 5th-generation tensor core
  return d;
}

// instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both operands K-major
__device__ __forceinline__ uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(MIX_TM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared bulk copy (16-byte aligned, multiple of 16 bytes), completion
// counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ uint16_t bf_bits(__nv_bfloat16 x) { return __bfloat16_as_ushort(x); }

// error-free sum of two floats (TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// double-float value (hi + lo) as three BF16 planes
__device__ __forceinline__ void split3(float a0, float a1, uint16_t& h, uint16_t& m, uint16_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(a0);
  const float r = (a0 - __bfloat162float(bh)) + a1;
  const __nv_bfloat16 bm = __float2bfloat16_rn(r);
  const __nv_bfloat16 bl = __float2bfloat16_rn(r - __bfloat162float(bm));
  h = bf_bits(bh);
  m = bf_bits(bm);
  l = bf_bits(bl);
}

// two 32-lane x 8-column loads and the wait, in one statement
__device__ __forceinline__ void tmem_ld2x8(uint32_t t0, uint32_t t1, float* v0, float* v1) {
  uint32_t a[8], b[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
        "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7])
      : "r"(t0), "r"(t1)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v0[i] = __uint_as_float(a[i]);
    v1[i] = __uint_as_float(b[i]);
  }
}

// two 32-lane x 8-column stores and the wait, in one statement
__device__ __forceinline__ void tmem_st2x8(uint32_t t0, uint32_t t1, const float* v0, const float* v1) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%16], {%0,%1,%2,%3,%4,%5,%6,%7};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%17], {%8,%9,%10,%11,%12,%13,%14,%15};\n\t"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(__float_as_uint(v0[0])),
      "r"(__float_as_uint(v0[1])), "r"(__float_as_uint(v0[2])), "r"(__float_as_uint(v0[3])),
      "r"(__float_as_uint(v0[4])), "r"(__float_as_uint(v0[5])), "r"(__float_as_uint(v0[6])),
      "r"(__float_as_uint(v0[7])), "r"(__float_as_uint(v1[0])), "r"(__float_as_uint(v1[1])),
      "r"(__float_as_uint(v1[2])), "r"(__float_as_uint(v1[3])), "r"(__float_as_uint(v1[4])),
      "r"(__float_as_uint(v1[5])), "r"(__float_as_uint(v1[6])), "r"(__float_as_uint(v1[7])), "r"(t0), "r"(t1)
      : "memory");
}

// Persistent split-BF16 grouped GEMM.  Grid = min(#tiles, #SMs); CTA c takes the
// tiles c, c + G, c + 2G, ... of a list sorted by decreasing work.  18 warps (at
// most five per SM sub-partition, so 96 registers each):
//   warp 0        TMEM allocation and the MMA issuer (one lane)
//   warp 1        producer: plan records, tile slots and bulk copies into the ring
//   warps 2-17    drain + epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 and
//                 columns 32 ((w - 2) / 4) .. +31 of each accumulator chunk
// The accumulators are double-buffered per chunk of CHUNK stages: buffer b holds
// acc0 (hi x hi) in TMEM columns [256 b, 256 b + 128) and acc1 (the five small
// products) in [256 b + 128, 256 b + 256); while the drain warps fold chunk g
// into their double-float register sums the MMA warp fills the other buffer.
__global__ void __maxnreg__(96)
    mixed_gemm_kernel(const MixTile* __restrict__ tiles, int ntiles, const MixProb* __restrict__ probs,
                      const MixSeg* __restrict__ segs, const int64_t* __restrict__ bcol,
                      const int64_t* __restrict__ ccol, const float* __restrict__ acol, int* err,
                      int* next_tile, int tn) {
  extern __shared__ __align__(1024) uint8_t smem[];
  TileSlot* slots = reinterpret_cast<TileSlot*>(smem + SLOT_OFF);
  StageInfo* info = reinterpret_cast<StageInfo*>(smem + INFO_OFF);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BAR_OFF);
  // bars: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], mma_fin, slot_full[2], slot_empty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 9);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;

  auto full = [&](int s) { return saddr(&bars[s]); };
  auto empty = [&](int s) { return saddr(&bars[STAGES + s]); };
  auto acc_full = [&](int b) { return saddr(&bars[2 * STAGES + b]); };
  auto acc_empty = [&](int b) { return saddr(&bars[2 * STAGES + 2 + b]); };
  const uint32_t mma_fin = saddr(&bars[2 * STAGES + 4]);
  auto slot_full = [&](int b) { return saddr(&bars[2 * STAGES + 5 + b]); };
  auto slot_empty = [&](int b) { return saddr(&bars[2 * STAGES + 7 + b]); };

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), DRAIN_THREADS / 32);
      mbar_init(slot_full(b), 1);
      mbar_init(slot_empty(b), DRAIN_THREADS / 32);
    }
    mbar_init(mma_fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---- MMA issuer: consumes the ring in order, driven by the stage control
    // words alone (no global loads on the tensor core's critical path)
    if (lane == 0) {
      int step = 0;      // global stage counter (ring position)
      int chunk = 0;     // global chunk counter (accumulator buffer rotation)
      int in_chunk = 0;
      uint32_t dbase = 0;
      for (;; ++step) {
        const int st = step % STAGES;
        if (!mbar_wait(full(st), (step / STAGES) & 1, abort_flag, err, 1)) goto mma_done;
        const StageInfo si = info[st];
        if (si.ksub == 0) break;
        if (in_chunk == 0) {
          const int b = chunk & 1, use = chunk >> 1;
          if (use > 0 && !mbar_wait(acc_empty(b), (use - 1) & 1, abort_flag, err, 4)) goto mma_done;
          dbase = tmem + 256u * b;
        }
        fence_after();
        const uint32_t id = idesc(si.nmma);
        const uint32_t base = saddr(smem + st * STAGE_BYTES);
        for (int kk = 0; kk < si.ksub; ++kk) {
          const uint32_t o = kk * 256;
          const uint64_t a0 = sdesc(base + o), a1 = sdesc(base + 512 + o), a2 = sdesc(base + 1024 + o);
          const uint64_t b0 = sdesc(base + OPER_BYTES + o), b1 = sdesc(base + OPER_BYTES + 512 + o),
                         b2 = sdesc(base + OPER_BYTES + 1024 + o);
          const uint32_t acc = (in_chunk == 0 && kk == 0) ? 0u : 1u;
          mma(dbase, a0, b0, id, acc);
          mma(dbase + 128, a0, b1, id, acc);
          mma(dbase + 128, a1, b0, id, 1u);
          mma(dbase + 128, a0, b2, id, 1u);
          mma(dbase + 128, a1, b1, id, 1u);
          mma(dbase + 128, a2, b0, id, 1u);
        }
        mma_commit(empty(st));
        if (++in_chunk == CHUNK || si.last) {
          mma_commit(acc_full(chunk & 1));
          in_chunk = 0;
          ++chunk;
        }
      }
      goto mma_end;
    mma_done:
      *abort_flag = 1;
      mma_commit(acc_full(chunk & 1));
    mma_end:
      // every MMA this thread issued has finished before TMEM is released
      mma_commit(mma_fin);
      mbar_wait_exit(mma_fin, 0, err);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- producer warp: the only role that reads the plan from global memory.
    // Per tile it fills a tile slot for the drain warps (problem fields, and for
    // gathered problems the column tables by bulk copy); per stage it writes the
    // control word and copies the operand slabs: the slab of a 128-row operand
    // tile is contiguous in HBM (blocked split layout), so a stage is one bulk copy
    // for A and one for B (one per 8-row group for gathered A rows), completing on
    // the stage's transaction count.  The next tile's records are prefetched one
    // tile ahead.
    int step = 0, tcount = 0;
    bool stop = false;
    // CTA c starts with tile c.  With a counter (next_tile), each next tile is
    // claimed from it when the CTA starts the previous one, so tiles are handed out
    // in list order: tiles next to each other in the list share operand slabs (the
    // tiles of one output block) and start within a tile's claim of each other,
    // reading the shared slabs while the L2 still holds them.  Without one, CTA c
    // takes tiles c, c + G, c + 2G, ... (no atomic on the path of short tiles).
    int ti = blockIdx.x;
    MixTile t1{};
    MixProb p1{};
    MixSeg g1{};
    if (ti < ntiles) {
      t1 = tiles[ti];
      p1 = probs[t1.prob];
      if (p1.s1 > p1.s0) g1 = segs[p1.s0];
    }
    for (; ti < ntiles && !stop; ++tcount) {
      const MixTile tl = t1;
      const MixProb p = p1;
      const MixSeg gf = g1;
      int nx = ti + G;
      if (next_tile) {
        if (lane == 0) nx = G + atomicAdd(next_tile, 1);
        nx = __shfl_sync(0xffffffffu, nx, 0);
      }
      if (nx < ntiles) {
        t1 = tiles[nx];
        p1 = probs[t1.prob];
        if (p1.s1 > p1.s0) g1 = segs[p1.s0];
      }
      const int slot = tcount & 1;
      if (tcount >= 2 && !mbar_wait_warp(slot_empty(slot), ((tcount >> 1) - 1) & 1, abort_flag, err, 6)) {
        stop = true;
        break;
      }
      const int Nt = min(tn, p.N - tl.n0);
      if (lane == 0) {
        TileSlot& sl = slots[slot];
        sl.Chi = p.Chi;
        sl.Clo = p.Clo;
        sl.Cp = p.Cp;
        sl.m0 = tl.m0;
        sl.n0 = tl.n0;
        sl.Nt = Nt;
        sl.nch = (tl.nsteps + CHUNK - 1) / CHUNK;
        sl.M = p.M;
        sl.ldc = p.ldc;
        sl.mode = p.mode;
        sl.row0 = p.row0;
        sl.crows = p.crows;
        sl.alpha = p.alpha;
        sl.pad = 0;   // a tile (1 marks the sentinel)
        if (p.mode == 3) {
          const int Mt = min(MIX_TM, p.M - tl.m0);
          mbar_expect_tx(slot_full(slot), uint32_t(Mt) * 12u);
          bulk_copy(saddr(sl.c), ccol + p.cm0 + tl.m0, uint32_t(Mt) * 8u, slot_full(slot));
          bulk_copy(saddr(sl.a), acol + p.cm0 + tl.m0, uint32_t(Mt) * 4u, slot_full(slot));
        } else {
          mbar_arrive(slot_full(slot));
        }
      }
      const int hA = min(MIX_TM, ((p.M + 7) & ~7) - tl.m0);   // rows of A in the tile (multiple of 8)
      const int hB = min(tn, ((p.N + 7) & ~7) - tl.n0);
      // a tile narrower than 128 starts inside a 128-row block of B: its rows are a
      // contiguous run at row offset n0 % 128 of each slab, whose stride is set by
      // the block's height
      const int hBk = min(MIX_TN, ((p.N + 7) & ~7) - (tl.n0 & ~127));
      const int64_t u0 = p.cm0 / 8 + (tl.m0 >> 3);            // first gathered unit of the tile
      const int nmma = (Nt + 15) & ~15;
      int left = tl.nsteps;
      for (int s = p.s0; s < p.s1 && !stop; ++s) {
        const MixSeg g = (s == p.s0) ? gf : segs[s];
        const int64_t Kt = (g.K + 31) & ~31;
        const uint16_t* Ab = g.A + int64_t(tl.m0 >> 7) * 384 * Kt;
        const uint16_t* Bb = g.B + int64_t(tl.n0 >> 7) * 384 * Kt + (tl.n0 & 127) * 96;
        for (int k0 = 0; k0 < g.K; k0 += BK, ++step) {
          const int st = step % STAGES;
          if (step >= STAGES && !mbar_wait_warp(empty(st), ((step / STAGES) - 1) & 1, abort_flag, err, 2)) {
            stop = true;
            break;
          }
          const bool last = (--left == 0);
          const uint32_t base = saddr(smem + st * STAGE_BYTES);
          const int64_t sl = k0 >> 5;
          if (lane == 0) {
            info[st] = StageInfo{(g.K - k0 > 16) ? 2 : 1, last ? 1 : 0, nmma, 0};
            mbar_expect_tx(full(st), uint32_t(hA + hB) * 192u);
            if (p.mode != 3) bulk_copy(base, Ab + sl * 96 * hA, uint32_t(hA) * 192u, full(st));
            bulk_copy(base + OPER_BYTES, Bb + sl * 96 * hBk, uint32_t(hB) * 192u, full(st));
          }
          __syncwarp();   // the transaction count is raised before the gathered copies
          if (p.mode == 3 && lane < (hA >> 3)) {
            const int64_t b0 = bcol[2 * (u0 + lane)], bs = bcol[2 * (u0 + lane) + 1];
            bulk_copy(base + lane * RG_BYTES, g.A + b0 + sl * bs, RG_BYTES, full(st));
          }
        }
      }
      ti = nx;
    }
    if (!stop) {
      // sentinel tile slot: the drain warps stop at it
      const int slot = tcount & 1;
      if (tcount >= 2 && !mbar_wait_warp(slot_empty(slot), ((tcount >> 1) - 1) & 1, abort_flag, err, 6)) {
        stop = true;
      } else {
        if (lane == 0) {
          slots[slot].pad = 1;
          mbar_arrive(slot_full(slot));
        }
        ++tcount;
      }
    }
    if (!stop) {
      // end marker for the MMA issuer
      const int st = step % STAGES;
      if (step < STAGES || mbar_wait_warp(empty(st), ((step / STAGES) - 1) & 1, abort_flag, err, 2)) {
        if (lane == 0) {
          info[st] = StageInfo{0, 0, 0, 0};
          mbar_arrive(full(st));
        }
        ++step;
      }
    }
    // no copy into this CTA's shared memory may still be in flight at exit: wait for
    // the last issued stages and tile slots (already complete unless a role aborted)
    if (lane == 0) {
      for (int s = max(0, step - STAGES); s < step; ++s) mbar_wait_exit(full(s % STAGES), (s / STAGES) & 1, err);
      for (int t = max(0, tcount - 2); t < tcount; ++t) mbar_wait_exit(slot_full(t & 1), (t >> 1) & 1, err);
    }
    __syncwarp();
  } else {
    // ---- drain + epilogue.  After an abort every wait returns at once; TMEM
    // contents are then meaningless but every store still goes to the addresses of
    // a tile slot that did arrive, and the tile loop ends at the next check.
    const int dw = warp - 2;                     // 0..15
    const int ch = dw >> 2;                      // column quarter: [32 ch, 32 ch + 32)
    const int row = (warp & 3) * 32 + lane;      // TMEM lane quarter = warp % 4
    const uint32_t tq = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + uint32_t(DRAIN_COLS * ch);
    int chunk = 0, tcount = 0;
    for (;; ++tcount) {
      const int slot = tcount & 1;
      if (!mbar_wait_warp(slot_full(slot), (tcount >> 1) & 1, abort_flag, err, 7)) break;
      const TileSlot& S = slots[slot];
      if (S.pad) break;   // the sentinel: no more tiles for this CTA
      const int nch = S.nch;
      const bool mine = DRAIN_COLS * ch < S.Nt;  // this warp's columns exist in the tile
      // running sum per element: sh + sl, where sh collects the hi x hi chunks
      // exactly (TwoSum) and sl their rounding errors plus the small products,
      // which are 2^-8 of the result and need no more than FP32.  After the last
      // chunk the sums are parked in that chunk's accumulator columns (sh over
      // acc0, sl over acc1) and the epilogue streams them out of TMEM, so that no
      // more than eight columns are live in registers while it stores.
      {
        float sh[DRAIN_COLS], sl[DRAIN_COLS];
#pragma unroll
        for (int i = 0; i < DRAIN_COLS; ++i) sh[i] = sl[i] = 0.f;
        for (int c = 0; c < nch; ++c, ++chunk) {
          const int b = chunk & 1;
          mbar_wait_warp(acc_full(b), (chunk >> 1) & 1, abort_flag, err, 3);
          fence_after();
          const uint32_t t0 = tq + 256u * b;
          // a tile of one chunk is its own running sum: sh = acc0 and sl = acc1
          // exactly, already in place for the epilogue (nch is tile-uniform)
          if (mine && nch > 1) {
#pragma unroll
            for (int h = 0; h < DRAIN_COLS / 8; ++h) {
              float v0[8], v1[8];
              tmem_ld2x8(t0 + 8 * h, t0 + 128 + 8 * h, v0, v1);
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                float s, e;
                two_sum(sh[8 * h + i], v0[i], s, e);
                sh[8 * h + i] = s;
                sl[8 * h + i] += e + v1[i];
              }
              if (c == nch - 1) tmem_st2x8(t0 + 8 * h, t0 + 128 + 8 * h, sh + 8 * h, sl + 8 * h);
            }
          }
          if (c < nch - 1) {
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty(b));
          }
        }
      }
      // epilogue: this thread owns row `row`, columns n0 + 32 ch + i.  The TMEM
      // loads are warp-collective (.sync.aligned), so they run under the
      // warp-uniform `mine` alone and rows past M only skip their stores.
      const int gm = S.m0 + row;
      const bool live = gm < S.M;
      const int cbase = DRAIN_COLS * ch;
      const uint32_t tl = tq + 256u * uint32_t((chunk - 1) & 1);   // parked sums (nch > 0)
      if (mine) {
        const float alpha = S.alpha;
        if (S.mode == 0) {
          float* Chi = S.Chi;
          float* Clo = S.Clo;
          const int64_t o0 = int64_t(gm) * S.ldc + S.n0 + cbase;
          const int nloc = min(DRAIN_COLS, S.Nt - cbase);
#pragma unroll
          for (int h = 0; h < DRAIN_COLS / 8; ++h) {
            float v0[8], v1[8];
            if (nch > 0) {
              tmem_ld2x8(tl + 8 * h, tl + 128 + 8 * h, v0, v1);
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) v0[i] = v1[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if (live && 8 * h + i < nloc) {
                float hi, lo;
                two_sum(alpha * v0[i], alpha * v1[i], hi, lo);
                Chi[o0 + 8 * h + i] = hi;
                Clo[o0 + 8 * h + i] = lo;
              }
            }
          }
        } else {
          // modes 2 and 3: tile row gm is row r of the blocked split matrix C (mode
          // 2: r = row0 + gm; mode 3: row part and row-block height from the
          // table) and this thread's 32 columns are one K slab of it, so each of
          // the three planes is four aligned 16-byte runs
          int64_t rowpart = 0;
          int h8 = 0;
          float al = alpha;
          bool store = live;
          if (S.mode == 3) {
            const int64_t e = live ? S.c[gm - S.m0] : -1;
            store = e >= 0;
            rowpart = e & ((int64_t(1) << 48) - 1);
            h8 = 8 * int(e >> 48);
            al = live ? S.a[gm - S.m0] : 0.f;
          } else if (live) {
            const int r = S.row0 + gm, rb = r >> 7, rr = r & 127;
            h8 = min(128, S.crows - (rb << 7));
            rowpart = int64_t(rb) * 384 * S.ldc + (rr >> 3) * 768 + (rr & 7) * 8;
          }
          uint16_t* dst = S.Cp + rowpart + int64_t((S.n0 + cbase) >> 5) * 96 * h8;
#pragma unroll
          for (int j = 0; j < DRAIN_COLS / 8; ++j) {
            float v0[8], v1[8];
            if (nch > 0) {
              tmem_ld2x8(tl + 8 * j, tl + 128 + 8 * j, v0, v1);
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) v0[i] = v1[i] = 0.f;
            }
            uint32_t hw[4], mw[4], lw[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              uint16_t hh[2], mm[2], ll[2];
#pragma unroll
              for (int v = 0; v < 2; ++v) {
                float hi, lo;
                two_sum(al * v0[2 * u + v], al * v1[2 * u + v], hi, lo);
                split3(hi, lo, hh[v], mm[v], ll[v]);
              }
              hw[u] = hh[0] | (uint32_t(hh[1]) << 16);
              mw[u] = mm[0] | (uint32_t(mm[1]) << 16);
              lw[u] = ll[0] | (uint32_t(ll[1]) << 16);
            }
            if (store) {
              *reinterpret_cast<uint4*>(dst + 64 * j) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *reinterpret_cast<uint4*>(dst + 256 + 64 * j) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
              *reinterpret_cast<uint4*>(dst + 512 + 64 * j) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        if (nch > 0) mbar_arrive(acc_empty((chunk - 1) & 1));
        mbar_arrive(slot_empty(slot));
      }
      if (*abort_flag) break;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

__global__ void split_kernel(const SplitTask* __restrict__ t, int nt) {
  for (int i = blockIdx.x; i < nt; i += gridDim.x) {
    const SplitTask s = t[i];
    const int n = s.rows * s.cols;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int r = e / s.cols, c = e - r * s.cols;
      const double x = s.src[int64_t(r) * s.ld + c];
      const __nv_bfloat16 h = __double2bfloat16(x);
      const double r1 = x - static_cast<double>(__bfloat162float(h));
      const __nv_bfloat16 m = __double2bfloat16(r1);
      const double r2 = r1 - static_cast<double>(__bfloat162float(m));
      const __nv_bfloat16 l = __double2bfloat16(r2);
      if (s.dn) {
        uint16_t* d = s.dn + blk_off(0, s.rn0 + r, s.cn0 + c, s.rn8, s.ktn);
        d[0] = bf_bits(h);
        d[256] = bf_bits(m);
        d[512] = bf_bits(l);
      }
      if (s.dt) {
        uint16_t* d = s.dt + blk_off(0, s.rt0 + c, s.ct0 + r, s.rt8, s.ktt);
        d[0] = bf_bits(h);
        d[256] = bf_bits(m);
        d[512] = bf_bits(l);
      }
    }
  }
}

// sigma = sum over split-K parts p (fixed order) of the double-float partials
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nparts, int64_t n, float* hi, float* lo,
                                    int accumulate) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float sh = part[i], sl = part[n + i];
    if (accumulate) {
      float s, e;
      two_sum(hi[i], sh, s, e);
      e += lo[i] + sl;
      sh = s + e;
      sl = e - (sh - s);
    }
    for (int q = 1; q < nparts; ++q) {
      const float* pq = part + int64_t(q) * 2 * n;
      float s, e;
      two_sum(sh, pq[i], s, e);
      e += sl + pq[n + i];
      sh = s + e;
      sl = e - (sh - s);
    }
    hi[i] = sh;
    lo[i] = sl;
  }
}

__global__ void df_to_f64_kernel(const float* __restrict__ hi, const float* __restrict__ lo, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = static_cast<double>(hi[i]) + static_cast<double>(lo[i]);
}

}  // namespace

void launch_mixed_gemm(const MixTile* tiles, int ntiles, const MixProb* probs, const MixSeg* segs,
                       const int64_t* bcol, const int64_t* ccol, const float* acol, int* err, int* next_tile,
                       int tn, int nsm, cudaStream_t st) {
  // the shared-memory opt-in is a per-device attribute of the kernel: set it once
  // on every device that launches it (devices past 63 set it on every launch)
  static std::atomic<uint64_t> attr_set{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t bit = (dev >= 0 && dev < 64) ? (uint64_t(1) << dev) : 0;
  if (!bit || !(attr_set.load(std::memory_order_relaxed) & bit)) {
    if (cudaFuncSetAttribute(mixed_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) ==
        cudaSuccess)
      attr_set.fetch_or(bit, std::memory_order_relaxed);
  }
  const int grid = ntiles < nsm ? ntiles : nsm;
  if (ntiles > 0) {
    if (next_tile) cudaMemsetAsync(next_tile, 0, sizeof(int), st);
    mixed_gemm_kernel<<<grid, NTHREADS, SMEM_BYTES, st>>>(tiles, ntiles, probs, segs, bcol, ccol, acol, err, next_tile,
                                                          tn);
  }
}

void launch_split(const SplitTask* t, int ntask, cudaStream_t st) {
  if (ntask > 0) split_kernel<<<ntask < 65535 ? ntask : 65535, 256, 0, st>>>(t, ntask);
}

void launch_reduce_parts(const float* part, int nparts, int64_t n, float* hi, float* lo, int accumulate, int grid,
                         cudaStream_t st) {
  if (n > 0) reduce_parts_kernel<<<grid, 256, 0, st>>>(part, nparts, n, hi, lo, accumulate);
}

void launch_df_to_f64(const float* hi, const float* lo, double* out, int64_t n, int grid, cudaStream_t st) {
  if (n > 0) df_to_f64_kernel<<<grid, 256, 0, st>>>(hi, lo, out, n);
}

}  // namespace dmrg
