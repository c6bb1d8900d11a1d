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
// stages): after each chunk they are drained into a double-float running sum
// (hi + lo, TwoSum) kept in TMEM columns [256, 512).
//
// CTA = 9 warps.  Warp 0 allocates TMEM and one elected lane issues the MMAs;
// warps 1-4 load operand tiles (16-byte vector loads into the canonical
// no-swizzle K-major core-matrix layout); warps 5-8 drain the accumulators and
// run the epilogue.  A ring of four shared-memory stages is guarded by
// mbarriers; every wait is bounded and sets an error word instead of hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mixed.h"

namespace dmrg {
namespace {

constexpr int BK = 32;                          // K elements per stage
constexpr int STAGES = 4;
constexpr int PLANE_BYTES = MIX_TM * BK * 2;    // one 128 x 32 BF16 plane: 8 KiB
constexpr int STAGE_BYTES = 6 * PLANE_BYTES;    // 3 A planes + 3 B planes
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + BAR_BYTES;
constexpr int PRODUCER_WARPS = 3;
constexpr int PRODUCER_THREADS = 32 * PRODUCER_WARPS;
constexpr int DRAIN_THREADS = 256;              // 8 warps: 4 lane quarters x 2 column halves
constexpr int NTHREADS = 32 + PRODUCER_THREADS + DRAIN_THREADS;
constexpr int CHUNK = 4;                        // K stages per accumulator chunk (128 K)
constexpr int LAG = 2;                          // stages a producer keeps in flight before retiring one
constexpr long long WAIT_CYCLES = 4000000000LL; // about 2 s at 2 GHz
constexpr uint32_t TMEM_COLS = 512;

static_assert(MIX_TN == MIX_TM, "B tile uses the A plane size");

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

// bounded wait: gives up after WAIT_CYCLES or when another role aborted
__device__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* err, int code) {
  if (mbar_try(a, parity)) return true;
  const long long t0 = clock64();
  for (unsigned spin = 1;; ++spin) {
    if (mbar_try(a, parity)) return true;
    if ((spin & 255u) == 0) {
      if (*abort_flag) return false;
      if (clock64() - t0 > WAIT_CYCLES) {
        *abort_flag = 1;
        atomicExch(err, code);
        return false;
      }
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
// SBO = 512 B (next 8-row group along M/N, BK/8 core matrices per group)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((128u >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>(((BK / 8) * 128u >> 4) & 0x3FFFu) << 32;
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

// two 32-lane x 16-column loads (acc0 and acc1 chunks) and the wait, in one statement
__device__ __forceinline__ void tmem_ld2(uint32_t t0, uint32_t t1, float* v0, float* v1) {
  uint32_t a[16], b[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
        "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]),
        "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
        "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15])
      : "r"(t0), "r"(t1)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    v0[i] = __uint_as_float(a[i]);
    v1[i] = __uint_as_float(b[i]);
  }
}

__device__ __forceinline__ void tmem_st2(uint32_t t0, uint32_t t1, const float* v0, const float* v1) {
  uint32_t a[16], b[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    a[i] = __float_as_uint(v0[i]);
    b[i] = __float_as_uint(v1[i]);
  }
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%32], {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%33], {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31};\n\t"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(a[0]),
      "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]),
      "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(b[0]), "r"(b[1]), "r"(b[2]),
      "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]), "r"(b[10]), "r"(b[11]),
      "r"(b[12]), "r"(b[13]), "r"(b[14]), "r"(b[15]), "r"(t0), "r"(t1)
      : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
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

// Persistent split-BF16 grouped GEMM.  Grid = min(#tiles, #SMs); CTA c takes the
// tiles c, c + G, c + 2G, ... of a list sorted by decreasing work.  12 warps
// (three per SM sub-partition, so up to 168 registers each):
//   warp 0        TMEM allocation and the MMA issuer (one lane)
//   warps 1-3     producers: 16-byte loads of A/B planes into the smem ring
//   warps 4-11    drain + epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 and
//                 columns 64 ((w - 4) / 4) .. +63 of each accumulator chunk
// The accumulators are double-buffered per chunk of CHUNK stages: buffer b holds
// acc0 (hi x hi) in TMEM columns [256 b, 256 b + 128) and acc1 (the five small
// products) in [256 b + 128, 256 b + 256); while the drain warps fold chunk g
// into their double-float register sums the MMA warp fills the other buffer.
__global__ void __launch_bounds__(NTHREADS, 1)
    mixed_gemm_kernel(const MixTile* __restrict__ tiles, int ntiles, const MixProb* __restrict__ probs,
                      const MixSeg* __restrict__ segs, const int64_t* __restrict__ bcol,
                      const int64_t* __restrict__ ccol, const float* __restrict__ acol, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars: full[STAGES], empty[STAGES], acc_full[2], acc_empty[2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;

  auto full = [&](int s) { return saddr(&bars[s]); };
  auto empty = [&](int s) { return saddr(&bars[STAGES + s]); };
  auto acc_full = [&](int b) { return saddr(&bars[2 * STAGES + b]); };
  auto acc_empty = [&](int b) { return saddr(&bars[2 * STAGES + 2 + b]); };

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full(s), PRODUCER_WARPS);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full(b), 1);
      mbar_init(acc_empty(b), DRAIN_THREADS / 32);
    }
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
    // ---- MMA issuer
    if (lane == 0) {
      int step = 0;     // global stage counter (ring position)
      int chunk = 0;    // global chunk counter (accumulator buffer rotation)
      for (int ti = blockIdx.x; ti < ntiles; ti += G) {
        const MixTile tl = tiles[ti];
        const MixProb p = probs[tl.prob];
        const int Nt = min(MIX_TN, p.N - tl.n0);
        const uint32_t id = idesc((Nt + 15) & ~15);
        int in_chunk = 0;
        uint32_t dbase = 0;
        for (int s = p.s0; s < p.s1; ++s) {
          const int K = segs[s].K;
          for (int k0 = 0; k0 < K; k0 += BK, ++step) {
            if (in_chunk == 0) {
              const int b = chunk & 1, use = chunk >> 1;
              if (use > 0 && !mbar_wait(acc_empty(b), (use - 1) & 1, abort_flag, err, 4)) goto mma_done;
              dbase = tmem + 256u * b;
            }
            const int st = step % STAGES;
            if (!mbar_wait(full(st), (step / STAGES) & 1, abort_flag, err, 1)) goto mma_done;
            // the stage was written by cp.async (generic proxy); order it before the
            // tensor core's async-proxy reads
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_after();
            const uint32_t base = saddr(smem + st * STAGE_BYTES);
            const int ksub = (K - k0 > 16) ? 2 : 1;
            for (int kk = 0; kk < ksub; ++kk) {
              const uint32_t o = kk * 256;
              const uint64_t a0 = sdesc(base + o), a1 = sdesc(base + PLANE_BYTES + o),
                             a2 = sdesc(base + 2 * PLANE_BYTES + o);
              const uint64_t b0 = sdesc(base + 3 * PLANE_BYTES + o), b1 = sdesc(base + 4 * PLANE_BYTES + o),
                             b2 = sdesc(base + 5 * PLANE_BYTES + o);
              const uint32_t acc = (in_chunk == 0 && kk == 0) ? 0u : 1u;
              mma(dbase, a0, b0, id, acc);
              mma(dbase + 128, a0, b1, id, acc);
              mma(dbase + 128, a1, b0, id, 1u);
              mma(dbase + 128, a0, b2, id, 1u);
              mma(dbase + 128, a1, b1, id, 1u);
              mma(dbase + 128, a2, b0, id, 1u);
            }
            mma_commit(empty(st));
            if (++in_chunk == CHUNK) {
              mma_commit(acc_full(chunk & 1));
              in_chunk = 0;
              ++chunk;
            }
          }
        }
        if (in_chunk > 0) {
          mma_commit(acc_full(chunk & 1));
          ++chunk;
        }
      }
      goto mma_end;
    mma_done:
      *abort_flag = 1;
      mma_commit(acc_full(chunk & 1));
    mma_end:;
    }
    __syncwarp();
  } else if (warp < 1 + PRODUCER_WARPS) {
    // ---- producers
    const int pt = tid - 32;
    int step = 0;
    bool stop = false;
    for (int ti = blockIdx.x; ti < ntiles && !stop; ti += G) {
      const MixTile tl = tiles[ti];
      const MixProb p = probs[tl.prob];
      const int Nt = min(MIX_TN, p.N - tl.n0);
      const int Nmma = (Nt + 15) & ~15;
      for (int s = p.s0; s < p.s1 && !stop; ++s) {
        const MixSeg g = segs[s];
        const int Kp = (g.K + 7) & ~7;
        for (int k0 = 0; k0 < g.K; k0 += BK, ++step) {
          const int st = step % STAGES;
          if (step >= STAGES && !mbar_wait_warp(empty(st), ((step / STAGES) - 1) & 1, abort_flag, err, 2)) {
            stop = true;
            break;
          }
          const uint32_t base = saddr(smem + st * STAGE_BYTES);
          for (int idx = pt; idx < 512; idx += PRODUCER_THREADS) {
            const int r = idx >> 2, j = idx & 3;
            const int k = k0 + 8 * j;
            const uint32_t so = (((r >> 3) * (BK / 8) + j) << 7) + ((r & 7) << 4);
            const int gm = tl.m0 + r, gn = tl.n0 + r;
            const bool va = gm < p.M && k < Kp;
            const bool vb = r < Nmma && gn < p.N && k < Kp;
            // out-of-range chunks are zero-filled (source size 0, base pointer as a valid address)
            const uint16_t* a = va ? g.A + int64_t(gm) * g.lda + k : g.A;
            const uint16_t* bb =
                vb ? g.B + (p.mode == 3 ? bcol[p.cm0 + gn] : int64_t(gn) * g.ldb) + k : g.B;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              cp_async16(base + q * PLANE_BYTES + so, a + q * g.psA, va ? 16u : 0u);
              cp_async16(base + (3 + q) * PLANE_BYTES + so, bb + q * g.psB, vb ? 16u : 0u);
            }
          }
          // one commit group per stage; the stage issued LAG steps ago is retired when
          // its group has landed: the warp syncs and one lane arrives on its full barrier
          asm volatile("cp.async.commit_group;" ::: "memory");
          if (step >= LAG) {
            asm volatile("cp.async.wait_group %0;" ::"n"(LAG) : "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(full((step - LAG) % STAGES));
          }
        }
      }
    }
    // retire the last stages in order
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    if (lane == 0)
      for (int r = (step > LAG ? step - LAG : 0); r < step; ++r) mbar_arrive(full(r % STAGES));
  } else {
    // ---- drain + epilogue
    const int dw = warp - 1 - PRODUCER_WARPS;   // 0..7
    const int q4 = warp & 3;                     // TMEM lane quarter of this warp
    const int ch = dw >> 2;                      // column half: columns [64 ch, 64 ch + 64)
    const int row = q4 * 32 + lane;
    const uint32_t lane_off = static_cast<uint32_t>(q4 * 32) << 16;
    int chunk = 0;
    bool ok = true;
    for (int ti = blockIdx.x; ti < ntiles; ti += G) {
      const MixTile tl = tiles[ti];
      const MixProb p = probs[tl.prob];
      const int Nt = min(MIX_TN, p.N - tl.n0);
      const int Nmma = (Nt + 15) & ~15;
      int nsteps = 0;
      for (int s = p.s0; s < p.s1; ++s) nsteps += (segs[s].K + BK - 1) / BK;
      const int nch = (nsteps + CHUNK - 1) / CHUNK;
      float sh[64], sl[64];
#pragma unroll
      for (int i = 0; i < 64; ++i) sh[i] = sl[i] = 0.f;
      const bool mine = 64 * ch < Nmma;          // this warp's columns exist in the tile
      for (int c = 0; c < nch; ++c, ++chunk) {
        const int b = chunk & 1, use = chunk >> 1;
        if (ok) ok = mbar_wait_warp(acc_full(b), use & 1, abort_flag, err, 3);
        fence_after();
        if (ok && mine) {
          const uint32_t t0 = tmem + lane_off + 256u * b + 64u * ch;
#pragma unroll
          for (int h = 0; h < 8; ++h) {
            float v0[8], v1[8];
            tmem_ld2x8(t0 + 8 * h, t0 + 128 + 8 * h, v0, v1);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float hi, lo;
              two_sum(v0[i], v1[i], hi, lo);
              float s, e;
              two_sum(sh[8 * h + i], hi, s, e);
              e += sl[8 * h + i] + lo;
              sh[8 * h + i] = s + e;
              sl[8 * h + i] = e - (sh[8 * h + i] - s);
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty(b));
      }
      // epilogue: this thread owns row `row`, columns n0 + 32 ch + i
      const int gm = tl.m0 + row;
      if (!mine || gm >= p.M) continue;
      const int cbase = 64 * ch;
      if (p.mode == 0) {
#pragma unroll
        for (int i = 0; i < 64; ++i) {
          if (cbase + i >= Nt) break;
          const int64_t o = int64_t(gm) * p.ldc + tl.n0 + cbase + i;
          float hi = p.alpha * sh[i], lo = p.alpha * sl[i];
          if (p.accumulate) {
            float s, e;
            two_sum(p.Chi[o], hi, s, e);
            e += p.Clo[o] + lo;
            hi = s + e;
            lo = e - (hi - s);
          }
          p.Chi[o] = hi;
          p.Clo[o] = lo;
        }
      } else if (p.mode == 1 && cbase + 64 <= Nt) {
        // 64 consecutive BF16 per plane as eight 16-byte stores (row starts and
        // column offsets are multiples of 8 elements in every plane layout)
        uint16_t* dst = p.Cp + int64_t(gm) * p.ldc + tl.n0 + cbase;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          uint32_t hw[4], mw[4], lw[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            uint16_t hh[2], mm[2], ll[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int c = 8 * v + 2 * i + u;
              split3(p.alpha * sh[c], p.alpha * sl[c], hh[u], mm[u], ll[u]);
            }
            hw[i] = hh[0] | (uint32_t(hh[1]) << 16);
            mw[i] = mm[0] | (uint32_t(mm[1]) << 16);
            lw[i] = ll[0] | (uint32_t(ll[1]) << 16);
          }
          reinterpret_cast<uint4*>(dst)[v] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          reinterpret_cast<uint4*>(dst + p.psC)[v] = make_uint4(mw[0], mw[1], mw[2], mw[3]);
          reinterpret_cast<uint4*>(dst + 2 * p.psC)[v] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      } else {
        // mode 1 tail, mode 2 (transposed store: tile column n goes to row n of C) or
        // mode 3 (column n goes to the row of C given by its table entry)
#pragma unroll
        for (int i = 0; i < 64; ++i) {
          if (cbase + i >= Nt) break;
          const int n = tl.n0 + cbase + i;
          int64_t o;
          float al = p.alpha;
          if (p.mode == 3) {
            o = ccol[p.cm0 + n] + gm;
            al = acol[p.cm0 + n];
          } else {
            o = (p.mode == 2) ? int64_t(n) * p.ldc + gm : int64_t(gm) * p.ldc + n;
          }
          uint16_t h, m, l;
          split3(al * sh[i], al * sl[i], h, m, l);
          p.Cp[o] = h;
          p.Cp[o + p.psC] = m;
          p.Cp[o + 2 * p.psC] = l;
        }
      }
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
        uint16_t* d = s.dn + int64_t(r) * s.ldn + c;
        d[0] = bf_bits(h);
        d[s.ps] = bf_bits(m);
        d[2 * s.ps] = bf_bits(l);
      }
      if (s.dt) {
        uint16_t* d = s.dt + int64_t(c) * s.ldt + r;
        d[0] = bf_bits(h);
        d[s.ps] = bf_bits(m);
        d[2 * s.ps] = bf_bits(l);
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
                       const int64_t* bcol, const int64_t* ccol, const float* acol, int* err, int nsm,
                       cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mixed_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    attr = true;
  }
  const int grid = ntiles < nsm ? ntiles : nsm;
  if (ntiles > 0) mixed_gemm_kernel<<<grid, NTHREADS, SMEM_BYTES, st>>>(tiles, ntiles, probs, segs, bcol, ccol, acol, err);
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
