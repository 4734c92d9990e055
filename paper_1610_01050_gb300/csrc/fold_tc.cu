// permute_window_fold on the tensor cores, for row chunks of 64 complex columns.
//
// Per residue class the fold of a loop group is a small dense contraction (see fold.cu for
// the source-order form): with X_r the 128 reals (re, im interleaved) of row r of the
// class and w_{r,l} = c + jd the row weight of loop l,
//     D1[m][l] = sum_r X_r[m] c_{r,l},   D2[m][l] = sum_r X_r[m] d_{r,l},
//     acc_l(col) = (D1[2col] - D2[2col+1]) + j (D1[2col+1] + D2[2col]),
// i.e. one real GEMM D[128 x 32] = A[128 x R] B[R x 32] per class with A = X^T and the
// first 2 LG columns of B holding (c, d).  tcgen05.mma kind::tf32 runs it with A and the
// accumulator in tensor memory and B in shared memory; FP32 accuracy comes from the
// three-term split A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi with hi = the operand rounded to
// the nearest TF32 value and lo = operand - hi (exact in FP32, then itself rounded to TF32:
// the tensor core would truncate it), which leaves 2^-22 of each product.  A tensor-core
// instruction at M = 128 takes the same time for any N up to 256, so the instruction count
// (two per 8 rows of a class) sets the kernel's floor and the N halves are free.  The high-low products share one instruction:
// A_hi x [B_hi | B_lo] (N = 64, the two B parts adjacent in shared memory) accumulates hh in
// TMEM columns [0, 32) and hl in [32, 64); then A_lo x B_hi (N = 32) adds lh to [0, 32).  The
// epilogue applies the column weights and sums the columns of equal residue in a fixed order
// (deterministic).
//
// Persistent CTAs (one per SM, 14 warps) walk units of two classes, warp-specialised:
//   * a producer warp streams each stage -- 16 rows of both classes, one tensor-map box --
//     through a ring of up to 12 slots;
//   * eight transposer warps (four per class; TMEM lane m = real column m) read the stage's
//     rows from the ring, split them into TF32 high and low parts and store them as the A
//     operand into one of four TMEM stage buffers (tcgen05.st), and write the stage's B
//     tiles (K-major core matrices of 8 rows x 16 bytes) into shared memory from the row
//     weights a_{l,in}(s_in) a_{l,out}(s_out), multiplied out of the per-dimension
//     residue-class tables (read through L1, prefetched a unit ahead);
//   * one thread of the MMA warp issues the stage's 8 MMAs and commits them to the stage
//     buffer's barrier, and at the end of a unit to the accumulator set's barrier;
//   * the epilogue warpgroup reads a unit's accumulators (two TMEM sets, so the next unit
//     accumulates meanwhile), applies the column weights and writes the buckets.
// Every wait is bounded; a wait that gives up sets the plan's error flag and the CTA's abort
// flag, and the other roles skip their remaining work.
#include <cuda.h>

#include "device.cuh"
#include "tma.cuh"

namespace rsft {
namespace {

constexpr int kTcClasses = 2;                        // classes per unit
constexpr int kTcRows = 16;                          // rows of each class per stage (two K steps)
constexpr int kTcW = 64;                             // complex columns per row
constexpr int kTcM = 2 * kTcW;                       // 128 reals: the MMA's M
constexpr int kTcN = 32;                             // B rows per part: (Re w, Im w) of <= 16 loops
constexpr int kTileB = kTcN * 8 * 4;                 // one B part (32 x 8 FP32): 1 KB
constexpr int kXBytes = kTcRows * kTcClasses * kTcM * 4;   // 16 KB of data per stage
constexpr int kBSet = 2 * kTileB;                    // B_hi, B_lo of one (class, K step)
constexpr int kBBuf = kTcClasses * 2 * kBSet;        // 8 KB of B per stage
constexpr int kRingMax = 12;                         // TMA stages in flight (at most)
constexpr int kStageBufs = 4;                        // A (TMEM) + B (shared) stage buffers
constexpr int kAccCols = 64;                         // TMEM columns per class: [0, 32) hh + lh, [32, 64) hl
constexpr int kAccSet = kTcClasses * kAccCols;       // 128 columns per accumulator set
constexpr int kACols = kTcClasses * 2 * kTcRows;     // 64 TMEM columns of A per stage: [class][hi, lo][16 rows]
constexpr int kABase = 2 * kAccSet;                  // A buffers after the two accumulator sets
constexpr int kTmemCols = kABase + kStageBufs * kACols;  // 512: the whole tensor memory
// warp roles: the epilogue warpgroup first (warp w reads TMEM lanes 32 (w % 4) ...)
constexpr int kEpiWarps = 4;
constexpr int kProducerWarp = 4;
constexpr int kMmaWarp = 5;
constexpr int kSplitWarp0 = 6, kSplitWarps = 8;
constexpr int kSplitThreads = 32 * kSplitWarps;
constexpr int kTcThreads = 32 * (kSplitWarp0 + kSplitWarps);  // 448
constexpr int kSmemMax = 227 * 1024;

struct TcArgs {
  CUtensorMap tmap;        // box: 64 complex columns x 2 classes x 16 rows (uint64 elements)
  int tensor_rank;         // 3 or 5
  Geometry g;
  FoldSchedule fs;
  int loop0, loops;        // first loop of the group, all loops of the plan (table stride)
  int units, nst, ring;    // units of two classes, stages per unit, ring slots
  int m_in, log_m_in, m_out, per_x;   // alias counts of the row dimensions; columns per residue
  int ring_off, b_off, colw_off, red_off, tab_off, bar_off;
  float2* folded;
  int* err;
  const float2* w_in;      // [B][L][M] weights of row dimension d_in - 1 by residue class
  const float2* w_out;     // the same of dimension 0 when there are two row dimensions
  const float2* colw;      // [lg][64] column weights (one column chunk)
  int jcol[kMaxLoopGroup * kTcW];  // [l][x] bucket offset of the column dimensions' residues
  int rsinv[kMaxLoopGroup * 2];    // [l][d] sigma^{-1} mod B_d of the row dimensions
  unsigned char colx[kTcW];        // the chunk's columns grouped by residue (per_x each, ascending)
};

// Float offset of element (r, k) in a K-major tile without swizzle: core matrix (r/8, k/4)
// holds 8 rows x 4 elements contiguously; K-adjacent core matrices 128 B apart (LBO), row
// groups 256 B apart (SBO).
__host__ __device__ __forceinline__ int kmajor(int r, int k) { return ((r >> 3) * 2 + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

__device__ __forceinline__ uint64_t operand_desc(const void* tile) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((smem_u32(tile) >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>(128 >> 4) << 16;  // leading byte offset: K-adjacent core matrices
  d |= static_cast<uint64_t>(256 >> 4) << 32;  // stride byte offset: 8-row groups
  d |= static_cast<uint64_t>(1) << 46;         // descriptor version
  return d;                                    // no swizzle, base offset 0
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands K-major.
__host__ __device__ constexpr uint32_t tf32_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

// x rounded to the nearest TF32 value (ties away from zero); x - tf32_rn(x) is exact in FP32
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// D (TMEM) (+)= A (TMEM, lane m = row m, column k) x B (shared memory descriptor)^T
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// 16 consecutive columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory"); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <int LG>
__global__ void __launch_bounds__(kTcThreads, 1) fold_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const Geometry& g = a.g;
  const FoldSchedule& fs = a.fs;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nst = a.nst, ring_n = a.ring;
  const int my_units = (a.units - static_cast<int>(blockIdx.x) + static_cast<int>(gridDim.x) - 1) /
                       static_cast<int>(gridDim.x);
  const int total = my_units * nst;

  unsigned char* ring = smem + a.ring_off;
  unsigned char* bbuf = smem + a.b_off;
  float2* colw = reinterpret_cast<float2*>(smem + a.colw_off);
  float2* red = reinterpret_cast<float2*>(smem + a.red_off);  // [class][64 columns][LG]
  int* s_jcol = reinterpret_cast<int*>(smem + a.tab_off);     // [LG][X]
  int* s_rsinv = s_jcol + LG * kTcW;                          // [LG][2]
  unsigned char* s_colx = reinterpret_cast<unsigned char*>(s_rsinv + 2 * LG);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.bar_off);  // [ring] stage landed
  uint64_t* empty = full + kRingMax;         // [ring] transposers done with the slot
  uint64_t* opfull = empty + kRingMax;       // [kStageBufs] A and B of a stage written
  uint64_t* opempty = opfull + kStageBufs;   // [kStageBufs] their MMAs retired
  uint64_t* accfull = opempty + kStageBufs;  // [2] a unit's accumulators complete
  uint64_t* accempty = accfull + 2;          // [2] the epilogue has read them
  uint64_t* cbar = accempty + 2;             // column weights landed
  uint64_t* drain = cbar + 1;                // every MMA retired (before TMEM is freed)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  if (tid == 0) {
    for (int i = 0; i < ring_n; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, kSplitWarps);
    }
    for (int i = 0; i < kStageBufs; ++i) {
      mbar_init(opfull + i, kSplitWarps);
      mbar_init(opempty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(accfull + i, 1);
      mbar_init(accempty + i, kEpiWarps);
    }
    mbar_init(cbar, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  // B rows 2 LG .. 31 of both parts stay zero (the per-stage writes never touch them)
  for (int e = tid; e < kStageBufs * kTcClasses * 2 * 2 * kTcN * 8; e += kTcThreads) {
    const int k = e & 7, n = (e >> 3) & (kTcN - 1), part = (e >> 8) & 1, set = (e >> 9) & 3, buf = e >> 11;
    if (n >= 2 * LG) {
      float* bt = reinterpret_cast<float*>(bbuf + buf * kBBuf + set * kBSet + part * kTileB);
      bt[kmajor(n, k)] = 0.f;
    }
  }
  // epilogue tables in shared memory (per-thread indexes of parameter arrays would serialise)
  for (int e = tid; e < LG * kTcW; e += kTcThreads) s_jcol[e] = a.jcol[e];
  for (int e = tid; e < 2 * LG; e += kTcThreads) s_rsinv[e] = a.rsinv[e];
  for (int e = tid; e < kTcW; e += kTcThreads) s_colx[e] = a.colx[e];
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (warp == kProducerWarp) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      const uint64_t pol_stream = policy_evict_first();
      const uint64_t pol_keep = policy_evict_last();
      mbar_arrive_expect_tx(cbar, static_cast<uint32_t>(LG * kTcW * 8));
      bulk_g2s(colw, a.colw, static_cast<uint32_t>(LG * kTcW * 8), cbar, pol_keep);
      for (int i = 0; i < total; ++i) {
        const int slot = i % ring_n;
        if (i >= ring_n && !mbar_wait(empty + slot, static_cast<uint32_t>(i / ring_n - 1) & 1u, abort_flag, a.err))
          break;
        const int u = static_cast<int>(blockIdx.x) + (i / nst) * static_cast<int>(gridDim.x);
        const int cls0 = u * kTcClasses, r0 = (i % nst) * kTcRows;
        unsigned char* dst = ring + slot * kXBytes;
        mbar_arrive_expect_tx(full + slot, static_cast<uint32_t>(kXBytes));
        if (a.tensor_rank == 3) {
          tensor_g2s_3d(dst, &a.tmap, 0, cls0 & static_cast<int>(g.b[0] - 1), r0, full + slot, pol_stream);
        } else {
          const int x1 = cls0 & static_cast<int>(g.b[1] - 1);
          const int x0 = (cls0 >> g.log_b[1]) & static_cast<int>(g.b[0] - 1);
          tensor_g2s_5d(dst, &a.tmap, 0, x1, r0 & static_cast<int>(g.m[1] - 1), x0, r0 >> g.log_m[1], full + slot,
                        pol_stream);
        }
      }
    }
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc_hl = tf32_idesc(kTcM, 2 * kTcN);  // A_hi x [B_hi | B_lo]
      constexpr uint32_t idesc_lh = tf32_idesc(kTcM, kTcN);      // A_lo x B_hi
      bool ok = true;
      int i = 0;
      for (int q = 0; q < my_units && ok; ++q) {
        const int ab = q & 1;
        if (q >= 2 && !mbar_wait(accempty + ab, static_cast<uint32_t>((q >> 1) - 1) & 1u, abort_flag, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int k = 0; k < nst; ++k, ++i) {
          const int b = i % kStageBufs;
          if (!mbar_wait(opfull + b, static_cast<uint32_t>(i / kStageBufs) & 1u, abort_flag, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const unsigned char* bb = bbuf + b * kBBuf;
          const uint32_t abuf = taddr + static_cast<uint32_t>(kABase + b * kACols);
#pragma unroll
          for (int c = 0; c < kTcClasses; ++c)
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) {
              const uint64_t bdesc = operand_desc(bb + (c * 2 + kb) * kBSet);
              const uint32_t d = taddr + static_cast<uint32_t>(ab * kAccSet + c * kAccCols);
              const uint32_t ahi = abuf + static_cast<uint32_t>(c * 2 * kTcRows + kb * 8);
              mma_ts(d, ahi, bdesc, idesc_hl, (k > 0 || kb > 0) ? 1 : 0);
              mma_ts(d, ahi + kTcRows, bdesc, idesc_lh, 1);
            }
          mma_commit(opempty + b);
        }
        if (!ok) break;
        mma_commit(accfull + ab);
      }
      // every MMA issued above retires before the TMEM is freed
      mma_commit(drain);
      mbar_wait_bounded(drain, 0u, a.err);
    }
  } else if (warp >= kSplitWarp0) {
    // ---------------------------------------------------------------- transposers
    const int st = tid - 32 * kSplitWarp0;
    const int cgrp = (warp - kSplitWarp0) >> 2;      // the class this warp transposes
    const int m = (warp & 3) * 32 + lane;            // its TMEM lane: real column m
    const uint32_t lanes = static_cast<uint32_t>((warp & 3) * 32) << 16;
    const int m_in = a.m_in, m_out = a.m_out, L = a.loops, l0 = a.loop0;
    const int din = fs.d_in;
    const int bin = static_cast<int>(g.b[din - 1]);
    bool ok = true;
    int i = 0;
    for (int q = 0; q < my_units && ok; ++q) {
      const int u = static_cast<int>(blockIdx.x) + q * static_cast<int>(gridDim.x);
      const int cls0 = u * kTcClasses;
      const int xo = din == 2 ? (cls0 >> g.log_b[1]) & static_cast<int>(g.b[0] - 1) : 0;
      const int xi0 = cls0 & (bin - 1);
      // the next unit's weight rows into L1 (a hint; the stage loads below read through L1)
      if (q + 1 < my_units) {
        const int cn = (u + static_cast<int>(gridDim.x)) * kTcClasses;
        const int xin = cn & (bin - 1);
        const int xon = din == 2 ? (cn >> g.log_b[1]) & static_cast<int>(g.b[0] - 1) : 0;
        const int in_bytes = LG * m_in * 8, out_bytes = din == 2 ? LG * m_out * 8 : 0;
        const int lines_in = (in_bytes + 127) >> 7, lines_out = (out_bytes + 127) >> 7;
        for (int e = st; e < 2 * lines_in + lines_out; e += kSplitThreads) {
          const char* p;
          if (e < 2 * lines_in) {
            const int c = e / lines_in;
            p = reinterpret_cast<const char*>(a.w_in + (static_cast<int64_t>(xin + c) * L + l0) * m_in) +
                (e % lines_in) * 128;
          } else {
            p = reinterpret_cast<const char*>(a.w_out + (static_cast<int64_t>(xon) * L + l0) * m_out) +
                (e - 2 * lines_in) * 128;
          }
          asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
        }
      }
      for (int k = 0; k < nst; ++k, ++i) {
        const int slot = i % ring_n, b = i % kStageBufs;
        // row weights of the stage: entry (class, K step, loop, row) -> w = a_in * a_out
        constexpr int kWE = kTcClasses * 2 * LG * 8;
        constexpr int kWPer = (kWE + kSplitThreads - 1) / kSplitThreads;
        float2 wv[kWPer];
#pragma unroll
        for (int t = 0; t < kWPer; ++t) {
          const int e = st + t * kSplitThreads;
          wv[t] = make_float2(0.f, 0.f);
          if (e < kWE) {
            const int kr = e & 7, l = (e >> 3) % LG, ckb = (e >> 3) / LG;
            const int c = ckb >> 1, kb = ckb & 1;
            const int r = k * kTcRows + kb * 8 + kr;
            const int mi = r & (m_in - 1), mo = r >> a.log_m_in;
            float2 w = __ldg(a.w_in + (static_cast<int64_t>(xi0 + c) * L + l0 + l) * m_in + mi);
            if (din == 2) w = cmul(w, __ldg(a.w_out + (static_cast<int64_t>(xo) * L + l0 + l) * m_out + mo));
            wv[t] = w;
          }
        }
        // the stage buffer's previous MMAs retired and the ring slot landed (warp-uniform:
        // the TMEM stores below are warp-collective)
        bool ready = i < kStageBufs ||
                     mbar_wait(opempty + b, static_cast<uint32_t>(i / kStageBufs - 1) & 1u, abort_flag, a.err);
        ready = ready && mbar_wait(full + slot, static_cast<uint32_t>(i / ring_n) & 1u, abort_flag, a.err);
        if (!__all_sync(0xffffffffu, ready)) {
          ok = false;
          break;
        }
        tc_fence_after();
        // A: this lane's real column over the stage's 16 rows of its class, split hi / lo
        const float* xs = reinterpret_cast<const float*>(ring + slot * kXBytes);
        float hi[kTcRows], lo[kTcRows];
#pragma unroll
        for (int r = 0; r < kTcRows; ++r) {
          const float x = xs[(r * kTcClasses + cgrp) * kTcM + m];
          hi[r] = tf32_rn(x);
          lo[r] = tf32_rn(x - hi[r]);
        }
        const uint32_t acol = taddr + lanes + static_cast<uint32_t>(kABase + b * kACols + cgrp * 2 * kTcRows);
        tmem_st16(acol, hi);
        tmem_st16(acol + kTcRows, lo);
        // B: rows l (Re w) and LG + l (Im w) of the high part, the same of the low part
        unsigned char* bb = bbuf + b * kBBuf;
#pragma unroll
        for (int t = 0; t < kWPer; ++t) {
          const int e = st + t * kSplitThreads;
          if (e < kWE) {
            const int kr = e & 7, l = (e >> 3) % LG, ckb = (e >> 3) / LG;
            float* bt = reinterpret_cast<float*>(bb + ckb * kBSet);
            const float2 w = wv[t];
            const float hr = tf32_rn(w.x), hm = tf32_rn(w.y);
            bt[kmajor(l, kr)] = hr;
            bt[kmajor(LG + l, kr)] = hm;
            bt[kTileB / 4 + kmajor(l, kr)] = tf32_rn(w.x - hr);
            bt[kTileB / 4 + kmajor(LG + l, kr)] = tf32_rn(w.y - hm);
          }
        }
        // A in TMEM and B visible to the tensor core, then the slot back to the producer
        // and the stage buffer to the MMA warp
        tmem_wait_st();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(empty + slot);
          mbar_arrive(opfull + b);
        }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue warpgroup
    const int X = fs.xcount, per_x = a.per_x;
    bool ok = mbar_wait(cbar, 0u, abort_flag, a.err);
    for (int q = 0; q < my_units; ++q) {
      const int u = static_cast<int>(blockIdx.x) + q * static_cast<int>(gridDim.x);
      const int cls0 = u * kTcClasses;
      const int ab = q & 1;
      if (ok && !mbar_wait(accfull + ab, static_cast<uint32_t>(q >> 1) & 1u, abort_flag, a.err)) ok = false;
      tc_fence_after();
      if (__all_sync(0xffffffffu, ok)) {  // tcgen05.ld and the shuffles need the whole warp
        const int m = warp * 32 + lane;
        const int col = m >> 1;
        const uint32_t lanes = static_cast<uint32_t>(warp * 32) << 16;
#pragma unroll
        for (int c = 0; c < kTcClasses; ++c) {
          uint32_t r[32], s[32];
          const uint32_t base = taddr + lanes + static_cast<uint32_t>(ab * kAccSet + c * kAccCols);
          tmem_ld32(base, r);
          tmem_ld32(base + kTcN, s);
          tmem_wait_ld();
#pragma unroll
          for (int l = 0; l < LG; ++l) {
            const float d1 = __uint_as_float(r[l]) + __uint_as_float(s[l]);
            const float d2 = __uint_as_float(r[LG + l]) + __uint_as_float(s[LG + l]);
            const float d1p = __shfl_xor_sync(0xffffffffu, d1, 1), d2p = __shfl_xor_sync(0xffffffffu, d2, 1);
            if ((lane & 1) == 0) {
              const float re = d1 - d2p, im = d1p + d2;
              const float2 w = colw[l * kTcW + col];
              red[(c * kTcW + col) * LG + l] = make_float2(w.x * re - w.y * im, w.x * im + w.y * re);
            }
          }
        }
      }
      // the accumulator set is free for the unit after next
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(accempty + ab);
      epi_barrier();
      if (ok) {
        for (int o = tid; o < kTcClasses * X * LG; o += 32 * kEpiWarps) {
          const int cc = o / (X * LG);
          const int rem = o - cc * X * LG;
          const int l = rem / X, x = rem - l * X;
          float2 sum = make_float2(0.f, 0.f);
          for (int j = 0; j < per_x; ++j) {
            const float2 v = red[(cc * kTcW + s_colx[x * per_x + j]) * LG + l];
            sum.x += v.x;
            sum.y += v.y;
          }
          // bucket j = sigma^{-1} x mod B per dimension (paper order): the column dimensions'
          // part from the table, the row dimensions' from the class residues
          const int cls = cls0 + cc;
          int64_t jb = s_jcol[l * X + x];
          if (fs.d_in == 2) {
            const int x1 = cls & static_cast<int>(g.b[1] - 1), x0 = (cls >> g.log_b[1]) & static_cast<int>(g.b[0] - 1);
            jb += static_cast<int64_t>((s_rsinv[l * 2] * x0) & static_cast<int>(g.b[0] - 1)) << g.b_shift[0];
            jb += static_cast<int64_t>((s_rsinv[l * 2 + 1] * x1) & static_cast<int>(g.b[1] - 1)) << g.b_shift[1];
          } else {
            const int x0 = cls & static_cast<int>(g.b[0] - 1);
            jb += static_cast<int64_t>((s_rsinv[l * 2] * x0) & static_cast<int>(g.b[0] - 1)) << g.b_shift[0];
          }
          a.folded[static_cast<int64_t>(a.loop0 + l) * g.total_b + jb] = sum;
        }
      }
      epi_barrier();  // the partials are read before the next unit writes them
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(kTmemCols) : "memory");
  }
}

// Shared memory of one CTA: ring slots, B stage buffers, column weights, epilogue partials
// and tables, barriers.  Returns the bytes; the ring takes what the rest leaves (<= 12 slots).
int tc_layout(int lg, int* ring, int* ring_off, int* b_off, int* colw_off, int* red_off, int* tab_off, int* bar_off) {
  const int fixed = kStageBufs * kBBuf + lg * kTcW * 8 + kTcClasses * kTcW * lg * 8 +
                    (lg * kTcW * 4 + 2 * lg * 4 + kTcW + 15) / 16 * 16 + (2 * kRingMax + 2 * kStageBufs + 6) * 8 + 16;
  int n = (kSmemMax - fixed) / kXBytes;
  *ring = n < kRingMax ? n : kRingMax;
  *ring_off = 0;
  *b_off = *ring * kXBytes;
  *colw_off = *b_off + kStageBufs * kBBuf;
  *red_off = *colw_off + lg * kTcW * 8;
  *tab_off = *red_off + kTcClasses * kTcW * lg * 8;
  *bar_off = *tab_off + (lg * kTcW * 4 + 2 * lg * 4 + kTcW + 15) / 16 * 16;
  return *bar_off + (2 * kRingMax + 2 * kStageBufs + 6) * 8 + 16;
}

using EncodeTiledFnTc = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFnTc encode_tiled_tc() {
  // looked up once; the initialisation of a function-local static is thread-safe
  static const EncodeTiledFnTc fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    EncodeTiledFnTc f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess && ptr)
      f = reinterpret_cast<EncodeTiledFnTc>(ptr);
    cudaGetLastError();
    return f;
  }();
  return fn;
}

// Tensor map of the stage boxes: dim 0 = a row's 64 complex columns (8-byte units), then for
// each row dimension (last first) its residue x_d and alias index m_d; the box spans two
// classes (consecutive x of the innermost row dimension) and 16 rows.  Rank 3 or 5, or 0.
int encode_tc_map(const Geometry& g, const FoldSchedule& fs, const float2* cube, CUtensorMap* map) {
  EncodeTiledFnTc fn = encode_tiled_tc();
  if (!fn || fs.d_in < 1 || fs.d_in > 2) return 0;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  dims[0] = static_cast<cuuint64_t>(fs.row_len);
  box[0] = kTcW;
  int rank = 1;
  int64_t sd = fs.row_len;
  int left = kTcRows;
  for (int d = fs.d_in - 1; d >= 0; --d) {
    const int64_t md = g.m[d];
    const int bm = static_cast<int>(left < md ? left : md);
    dims[rank] = static_cast<cuuint64_t>(g.b[d]);
    strides[rank - 1] = static_cast<cuuint64_t>(sd * 8);
    box[rank] = d == fs.d_in - 1 ? kTcClasses : 1u;
    ++rank;
    dims[rank] = static_cast<cuuint64_t>(md);
    strides[rank - 1] = static_cast<cuuint64_t>(sd * g.b[d] * 8);
    box[rank] = static_cast<cuuint32_t>(bm);
    ++rank;
    left /= bm;
    sd *= g.n[d];
  }
  if (left != 1) return 0;
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, static_cast<cuuint32_t>(rank), const_cast<float2*>(cube), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? rank : 0;
}

template <int LG>
cudaError_t launch_tc_lg(const TcArgs& args, int smem, cudaStream_t stream) {
  cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(fold_tc_kernel<LG>), smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = args.units < sms ? args.units : sms;  // one CTA per SM (all of its tensor memory)
  fold_tc_kernel<LG><<<grid, kTcThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace

bool fold_tc_supported(const Geometry& g, const FoldSchedule& fs) {
  if (fs.width != kTcW || fs.col_chunks != 1 || !fs.direct || fs.row_chunks != 1) return false;
  if (fs.lane_perm != 0x76543210u) return false;  // the epilogue tables assume thread = column pair
  if (fs.d_in < 1 || fs.d_in > 2 || fs.rows_per_chunk % kTcRows != 0 || fs.classes % kTcClasses != 0) return false;
  if (g.b[fs.d_in - 1] < kTcClasses) return false;  // the box's two classes are consecutive x_{d_in - 1}
  if (fs.xcount > kTcW || kTcW % fs.xcount != 0) return false;
  if (g.ndim - fs.d_in > 4) return false;
  // the tensor-map box: rows of a stage must tile the alias indices of the row dimensions
  int left = kTcRows;
  for (int d = fs.d_in - 1; d >= 0; --d) {
    const int64_t md = g.m[d];
    const int bm = static_cast<int>(left < md ? left : md);
    if (left % bm) return false;
    left /= bm;
  }
  if (left != 1) return false;
  const int lg = g.loops < kMaxLoopGroup ? g.loops : kMaxLoopGroup;
  int rn, ro, bo, co, rd, to, ba;
  return tc_layout(lg, &rn, &ro, &bo, &co, &rd, &to, &ba) <= kSmemMax && rn >= 4;
}

cudaError_t launch_fold_tc(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t, const float2* cube,
                           int loop0, int lg, float2* folded, int* err, int* copy_mode, cudaStream_t stream) {
  thread_local TcArgs args;
  args.tensor_rank = encode_tc_map(g, fs, cube, &args.tmap);
  if (copy_mode) *copy_mode = 100 + args.tensor_rank;
  if (args.tensor_rank == 0) return cudaErrorInvalidValue;
  args.g = g;
  args.fs = fs;
  args.loop0 = loop0;
  args.loops = g.loops;
  args.units = fs.classes / kTcClasses;
  args.nst = fs.rows_per_chunk / kTcRows;
  const int din = fs.d_in;
  args.m_in = static_cast<int>(g.m[din - 1]);
  args.log_m_in = g.log_m[din - 1];
  args.m_out = din == 2 ? static_cast<int>(g.m[0]) : 1;
  args.w_in = t.wcls[din - 1];
  args.w_out = din == 2 ? t.wcls[0] : t.wcls[din - 1];
  args.folded = folded;
  args.err = err;
  args.colw = t.fcolw + static_cast<int64_t>(loop0) * fs.col_chunks * fs.width;
  // bucket offsets: the column dimensions' part per (loop, residue), sigma^{-1} of the row dimensions
  for (int l = 0; l < lg; ++l) {
    for (int x = 0; x < fs.xcount; ++x) {
      int j = 0;
      for (int d = fs.d_in; d < g.ndim; ++d) {
        const int xd = t.h_xdig[x * 4 + (d - fs.d_in)];
        j += ((t.h_sinvb[(loop0 + l) * g.ndim + d] * xd) & static_cast<int>(g.b[d] - 1)) << g.b_shift[d];
      }
      args.jcol[l * fs.xcount + x] = j;
    }
    for (int d = 0; d < 2; ++d) args.rsinv[l * 2 + d] = d < fs.d_in ? t.h_sinvb[(loop0 + l) * g.ndim + d] : 0;
  }
  // columns grouped by residue, ascending within a residue (a fixed summation order)
  if (!t.h_xres) return cudaErrorInvalidValue;
  args.per_x = kTcW / fs.xcount;
  int fill[kTcW] = {0};
  for (int col = 0; col < kTcW; ++col) {
    const int x = t.h_xres[col];
    if (x >= fs.xcount || fill[x] >= args.per_x) return cudaErrorInvalidValue;
    args.colx[x * args.per_x + fill[x]++] = static_cast<unsigned char>(col);
  }
  const int smem = tc_layout(lg, &args.ring, &args.ring_off, &args.b_off, &args.colw_off, &args.red_off,
                             &args.tab_off, &args.bar_off);
  switch (lg) {
    case 1: return launch_tc_lg<1>(args, smem, stream);
    case 2: return launch_tc_lg<2>(args, smem, stream);
    case 3: return launch_tc_lg<3>(args, smem, stream);
    case 4: return launch_tc_lg<4>(args, smem, stream);
    case 5: return launch_tc_lg<5>(args, smem, stream);
    case 6: return launch_tc_lg<6>(args, smem, stream);
    case 7: return launch_tc_lg<7>(args, smem, stream);
    case 8: return launch_tc_lg<8>(args, smem, stream);
    case 9: return launch_tc_lg<9>(args, smem, stream);
    case 10: return launch_tc_lg<10>(args, smem, stream);
    case 11: return launch_tc_lg<11>(args, smem, stream);
    case 12: return launch_tc_lg<12>(args, smem, stream);
    case 13: return launch_tc_lg<13>(args, smem, stream);
    case 14: return launch_tc_lg<14>(args, smem, stream);
    case 15: return launch_tc_lg<15>(args, smem, stream);
    case 16: return launch_tc_lg<16>(args, smem, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rsft
