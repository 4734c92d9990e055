// permute_window_fold: the pre-window, permutation, flat window and aliasing
// steps of Algorithm 1 for a group of loops in one pass over the cube.
//
// Per loop l, Algorithm 1 computes f_l[j] = sum_{t = j mod B} w-bar(t) w(sigma t) r(sigma t)
// (eq. (l)).  With s = sigma t mod N (a bijection, Def. 1) this is
//     f_l[j] = sum_{s = x mod B} a_l(s) r(s),   j = sigma^{-1} x mod B,
//     a_l(s) = prod_d w-bar_d(sigma_d^{-1} s_d mod N_d) w_d(s_d),
// because t = j (mod B) iff s = sigma j (mod B) when B | N and sigma is odd.
// So the cube is read once, in its own order, and every element adds its
// weighted value to the bucket of its residue class x = s mod B in each loop;
// the permutation only selects the weight and relabels the B outputs.
//
// Work split (FoldSchedule): dimensions [0, d_in) index rows, [d_in, D) columns.
// A unit is C consecutive residue classes of the row dimensions (side by side), a
// chunk of their rows and a chunk of W columns.  Each thread keeps two fixed adjacent
// columns of one class and walks that class's rows, so its column weights factor out
// of the row loop:
//     acc_l(c) = sum_rows a_l^{row}(row) r(row, c),   contribution a_l^{col}(c) acc_l(c).
// A complex multiply-add w x r (w = c + jd, r = a + jb) is done with three real
// multiply-adds, K1 += c (a + b), K2 += (d - c) a, K3 += (c + d) b, and
// Re = K1 - K3, Im = K1 + K2 at the end; the row table holds (d - c, c + d, c, c) so that
// (K2, K3) of a column advance with one paired FP32 multiply-add on (a, b) as loaded, and the
// K1 of both columns with one more on the pair (a + b) of the two columns: no register moves
// to form operand pairs.
//
// Persistent CTAs (as many as fit, two per SM) walk the units.  TMA brings each
// stage of a shared-memory ring -- one tensor-map box holding a few rows of the C
// classes (or one 1-D bulk copy per row when rows are long) plus the matching slice
// of the row table -- and an mbarrier per slot signals its arrival; the last warp to
// finish with a slot refills it, so the next unit's rows arrive during an epilogue.
// The epilogue applies the column weights, sums threads of equal (class, residue)
// with warp shuffles over the lane bits that keep both, then across warps in a fixed
// order (deterministic results).  Which column pair a thread holds is a permutation of
// its index's bits chosen with the schedule: in chunk rows wider than a warp, lane bits
// 3-4 sit on column bits that keep the residue, so the shuffles do most of that sum.
// Every barrier wait is bounded in time; a wait that gives up sets the plan's error flag
// and the CTA skips its remaining work.
#include <cuda.h>

#include "device.cuh"
#include "tma.cuh"

namespace rsft {
namespace {

__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

constexpr int kThreads = kFoldConsumers;   // 256 threads, two columns each
static_assert(kThreads == 256, "fold_pair_of places 8 thread bits");
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRing = 8;                // shared-memory stages
constexpr int kStepsPerStage = kFoldStepsPerStage;  // row steps (2 * threads elements each) per stage
constexpr int kStepElems = 2 * kThreads;
constexpr int kStageBytes = kStepsPerStage * kStepElems * 8;
constexpr int kSmemBudget = 110 * 1024;    // two CTAs per SM

// Division by a launch constant: a shift and a mask when it is a power of two (all the fold's
// counts are for power-of-two geometries), else the plain operators.
struct Divisor {
  int d, s;  // s = log2 d, or -1
};
__host__ __device__ __forceinline__ Divisor divisor(int d) {
  Divisor v;
  v.d = d;
  v.s = -1;
  if (d > 0 && (d & (d - 1)) == 0) {
    v.s = 0;
    while ((1 << v.s) < d) ++v.s;
  }
  return v;
}
__device__ __forceinline__ int quo(int x, Divisor v) { return v.s >= 0 ? x >> v.s : x / v.d; }
__device__ __forceinline__ int rem(int x, Divisor v) { return v.s >= 0 ? x & (v.d - 1) : x % v.d; }

// The counts the stage issue divides by: stages per unit, units per frame, column chunks, row
// chunks, chunks per class group, ring slots.
struct IssueDivisors {
  Divisor nst, upf, cc, rc, ch, ring;
};

struct FoldArgs {
  CUtensorMap tmap[kMaxFrames];  // per frame: rows of C classes as one box (tensor mode)
  int tensor_rank;        // 0: one 1-D bulk copy per row; 3 or 5: one tensor copy per stage
  const float2* cube[kMaxFrames];
  int nframes;            // frames of one launch (units of frame f follow those of frame f - 1)
  int64_t folded_stride;  // elements between consecutive frames' folded buckets
  Geometry g;
  FoldSchedule fs;
  int loop0;
  int lg;
  int log_width;
  float2* folded;
  float2* partial;
  int* err;
  const float4* table;    // this loop group's row table: [group][row chunk][stage][row slot][step][record]
                          // (fold_record_f4 float4 a record; a row slot's records of one stage are adjacent)
  const float2* colw;     // this loop group's column weights: [col chunk][lg][W]
  int smem_colw;          // one column chunk: its weights staged in shared memory once
  int ring;               // stages in the ring
  int slot_bytes;         // data + the stage's row-table slice
  int colw_off, red_off, bar_off;             // shared-memory layout (bytes)
  int lch;                                    // loops per epilogue pass (the partials buffer holds lch loops)
  int sinvb[kMaxLoopGroup * kMaxDim];        // sigma^{-1} mod B_d of the group's loops
  unsigned short slots[512];                  // [C X][slots_per_x] epilogue partial sums per (class, residue)
  unsigned short xdig[2048];                  // [X][4] inner residue digits
  IssueDivisors dv;
  FoldClear clear;        // words zeroed by the grid before its work (detection bitmaps and counts)
};

// Stage geometry: a row step holds C classes x crow rows of W columns (rs = C crow rows);
// spst steps form a stage, nst stages a unit.
struct StageShape {
  int rs, spst, nst, data_bytes, table_bytes;
};

__host__ __device__ __forceinline__ StageShape stage_shape(const FoldSchedule& fs, int lg) {
  StageShape s;
  s.rs = fs.cps * fs.crow;
  s.spst = fold_stage_steps(fs);
  s.nst = fs.rows_per_chunk / fs.crow / s.spst;
  s.data_bytes = s.spst * s.rs * fs.width * 8;
  s.table_bytes = s.spst * s.rs * fold_record_f4(lg) * 16;
  return s;
}

// Column weights are staged once in shared memory when there is one column chunk and they
// fit in 16 KiB; otherwise the epilogue reads them through L1.
__host__ __device__ __forceinline__ bool colw_staged(const FoldSchedule& fs, int lg) {
  return fs.col_chunks == 1 && lg * fs.width * 8 <= 16 * 1024;
}

constexpr int kRedCap = 24 * 1024;  // epilogue partials: loops go through in passes of at most this

// Shared memory: [ring x (stage data | stage row table)] [column weights] [epilogue partials] [barriers].
// The partials hold lch loops at a time (all of them unless that would pass kRedCap).
__host__ __device__ __forceinline__ int fold_layout(const FoldSchedule& fs, int lg, int* ring, int* slot_bytes,
                                                    int* colw_off, int* red_off, int* bar_off, int* lch) {
  const StageShape sh = stage_shape(fs, lg);
  *slot_bytes = kStageBytes + sh.table_bytes;
  const int colw = colw_staged(fs, lg) ? lg * fs.width * 8 : 0;
  const int red_loop = kWarps * fs.leaders * 2 * 8;
  int lc = kRedCap / red_loop;
  if (lc < 1) lc = 1;
  if (lc > lg) lc = lg;
  *lch = lc;
  const int red = red_loop * lc;
  const int bars = (kMaxRing + 1) * 8 + kMaxRing * 4 + 16;
  int r = (kSmemBudget - colw - red - bars) / *slot_bytes;
  if (r > kMaxRing) r = kMaxRing;
  if (r < 2) r = 2;
  *ring = r;
  int off = r * *slot_bytes;
  *colw_off = off;
  off += colw;
  *red_off = off;
  off += red;
  *bar_off = off;
  off += bars;
  return off;
}

// Persistent fold: CTA b folds units b, b + grid, b + 2 grid, ... (a unit: C classes side by
// side, one row chunk, one column chunk).  The ring stays full across unit boundaries (the
// next unit's rows arrive during this unit's epilogue): the last warp to finish with stage i
// (a shared-memory count per slot) issues stage i + ring into the same slot.  Each stage
// brings its rows and their row-table slice.
// FULL: every row step fills the 2 * threads elements and every stage has kStepsPerStage steps,
// so the row-step strides are constants.
template <int LG, bool CHUNK, bool FULL>
__global__ void __launch_bounds__(kThreads, 2) fold_kernel(const __grid_constant__ FoldArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  chain_wait();
  chain_release();
  constexpr int NP = (LG + 1) / 2;        // float4 of (d - c, c + d) pairs in a row record (two loops each)
  constexpr int NC = (LG + 3) / 4;        // float4 of c values (four loops each)
  constexpr int REC = NP + NC;
  const Geometry& g = a.g;
  const FoldSchedule& fs = a.fs;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int R = fs.rows_per_chunk;
  const int W = fs.width;
  const int C = fs.cps;
  const StageShape sh = stage_shape(fs, LG);
  const int RS = sh.rs, spst = sh.spst, nst = sh.nst;
  const int ring = a.ring;
  const int chunks = fs.row_chunks * fs.col_chunks;
  const int units_pf = fs.groups * chunks;          // units of one frame
  const int units = units_pf * a.nframes;
  const int my_units = (units - static_cast<int>(blockIdx.x) + static_cast<int>(gridDim.x) - 1) /
                       static_cast<int>(gridDim.x);
  const int total = my_units * nst;  // stages of this CTA

  float2* colw = reinterpret_cast<float2*>(smem + a.colw_off);
  float2* red = reinterpret_cast<float2*>(smem + a.red_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + a.bar_off);
  uint64_t* cbar = full + kMaxRing;
  int* released = reinterpret_cast<int*>(cbar + 1);  // [ring] warps done with the slot's stage
  volatile int* abort_flag = released + kMaxRing;

  {
    // the next stage's detection bitmaps and counts start from zero
    const int64_t nthreads = static_cast<int64_t>(gridDim.x) * kThreads;
    for (int64_t w = static_cast<int64_t>(blockIdx.x) * kThreads + tid; w < a.clear.na; w += nthreads) a.clear.a[w] = 0u;
    for (int64_t w = static_cast<int64_t>(blockIdx.x) * kThreads + tid; w < a.clear.nb; w += nthreads) a.clear.b[w] = 0u;
  }
  if (tid == 0) {
    for (int i = 0; i < ring; ++i) {
      mbar_init(full + i, 1);
      released[i] = 0;
    }
    mbar_init(cbar, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();

  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  // Stage i of this CTA (one thread): unit blockIdx.x + (i / nst) grid, stage i % nst of it.  The
  // issuing thread holds up its warp, and the ring's next refill waits for that warp: keep it short.
  auto issue = [&](int i) {
    const IssueDivisors& dv = a.dv;
    const int uf = static_cast<int>(blockIdx.x) + quo(i, dv.nst) * static_cast<int>(gridDim.x);
    const int f = quo(uf, dv.upf), u = rem(uf, dv.upf);  // frame, unit within the frame
    const CUtensorMap* fmap = &a.tmap[f];                 // (the parameter block's own copy)
    const int k = rem(i, dv.nst);
    const int cc = rem(u, dv.cc);
    const int rc = rem(quo(u, dv.cc), dv.rc);
    const int grp = quo(u, dv.ch);
    const int cls0 = grp * C;     // first class of the unit
    const int slot = rem(i, dv.ring);
    unsigned char* base = smem + slot * a.slot_bytes;
    float2* dst = reinterpret_cast<float2*>(base);
    mbar_arrive_expect_tx(full + slot, static_cast<uint32_t>(sh.data_bytes + sh.table_bytes));
    const int r0 = rc * R + k * spst * fs.crow;  // first row (within each class) of the stage
    bulk_g2s(base + kStageBytes,
             a.table + ((static_cast<int64_t>(grp) * fs.row_chunks + rc) * R + k * spst * fs.crow) * C * REC,
             static_cast<uint32_t>(sh.table_bytes), full + slot, pol_keep);
    if (a.tensor_rank == 3) {
      tensor_g2s_3d(dst, fmap, cc * W, cls0 & static_cast<int>(g.b[0] - 1), r0, full + slot, pol_stream);
    } else if (a.tensor_rank == 5) {
      const int x1 = cls0 & static_cast<int>(g.b[1] - 1);
      const int x0 = (cls0 >> g.log_b[1]) & static_cast<int>(g.b[0] - 1);
      tensor_g2s_5d(dst, fmap, cc * W, x1, r0 & static_cast<int>(g.m[1] - 1), x0, r0 >> g.log_m[1], full + slot,
                    pol_stream);
    } else {
      for (int j = 0; j < spst * RS; ++j) {
        const int step = j / RS;
        const int ro = j - step * RS;
        int r = r0 + step * fs.crow + ro / C, c = cls0 + ro % C;
        int64_t row = 0, stride = 1;
#pragma unroll
        for (int d = kMaxDim - 1; d >= 0; --d) {
          if (d < fs.d_in) {
            const int xd = c & static_cast<int>(g.b[d] - 1);
            c >>= g.log_b[d];
            const int md = r & static_cast<int>(g.m[d] - 1);
            r >>= g.log_m[d];
            row += static_cast<int64_t>(xd + (md << g.log_b[d])) * stride;
            stride *= g.n[d];
          }
        }
        bulk_g2s(dst + step * RS * W + ro * W, a.cube[f] + row * fs.row_len + static_cast<int64_t>(cc) * W,
                 static_cast<uint32_t>(W * 8), full + slot, pol_stream);
      }
    }
  };
  const bool smem_colw = a.smem_colw != 0;
  if (tid == 0) {
    if (smem_colw) {
      mbar_arrive_expect_tx(cbar, static_cast<uint32_t>(LG * W * 8));
      bulk_g2s(colw, a.colw, static_cast<uint32_t>(LG * W * 8), cbar, pol_keep);
    }
    const int first = total < ring ? total : ring;
    for (int i = 0; i < first; ++i) issue(i);
  }

  // this thread: columns cp, cp + 1 of row slot ro = (class c = ro % C, row ro / C) of each step
  // (pair pq of the step: the thread's bits as the schedule places them)
  const int pq = fold_pair_of(tid, fs.lane_perm);
  const int cp = (2 * pq) & (W - 1);
  const int ro = (2 * pq) >> a.log_width;
  const bool active = ro < RS;
  bool ok = true;
  if (smem_colw) ok = mbar_wait(cbar, 0u, abort_flag, a.err);

  // epilogue constants
  const int nl = fs.leaders;
  const unsigned rmask = static_cast<unsigned>(fs.red_mask);
  const bool leader = (lane & rmask) == 0;
  int lj = 0;  // index of this leader among the warp's leaders (lane bits outside rmask, compressed)
  {
    int bit = 0;
#pragma unroll
    for (int b = 0; b < 5; ++b)
      if (!((rmask >> b) & 1u)) {
        lj |= ((lane >> b) & 1) << bit;
        ++bit;
      }
  }
  const int X = fs.xcount;
  const int keys = C * X;
  const int per = fs.slots_per_x;

  int slot = 0;
  uint32_t parity = 0u;
  int i = 0;  // stage counter
  for (int q = 0; q < my_units; ++q) {
    const int uf = static_cast<int>(blockIdx.x) + q * static_cast<int>(gridDim.x);
    const int frame = uf / units_pf, u = uf - frame * units_pf;
    float2* folded = a.folded + static_cast<int64_t>(frame) * a.folded_stride;
    const int cc = u % fs.col_chunks;
    const int rc = (u / fs.col_chunks) % fs.row_chunks;
    const int cls0 = (u / chunks) * C;
    // (K2, K3) of loop l for columns cp (k12a) and cp + 1 (k12b); K1 of loops 2p and 2p + 1 for
    // column cp (k1a[p]) and cp + 1 (k1b[p])
    float2 k12a[LG], k12b[LG], k1a[NP], k1b[NP];
#pragma unroll
    for (int l = 0; l < LG; ++l) {
      k12a[l] = make_float2(0.f, 0.f);
      k12b[l] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      k1a[q] = make_float2(0.f, 0.f);
      k1b[q] = make_float2(0.f, 0.f);
    }
    for (int k = 0; k < nst; ++k, ++i) {
      if (ok && !mbar_try_wait(full + slot, parity) && !mbar_wait(full + slot, parity, abort_flag, a.err)) ok = false;
      if (ok && active) {
        const float4* src = reinterpret_cast<const float4*>(smem + slot * a.slot_bytes) + pq;
        // this row slot's records of the stage's steps, one after another: (d - c, c + d) pairs of
        // two loops per float4, then c of four loops per float4
        const float4* tr =
            reinterpret_cast<const float4*>(smem + slot * a.slot_bytes + kStageBytes) + ro * (FULL ? kStepsPerStage : spst) * REC;
        const int dstride = FULL ? kStepElems / 2 : RS * W / 2;  // float4 from one row step to the next
#pragma unroll 2
        for (int step = 0; step < kStepsPerStage; ++step) {
          if (FULL || step < spst) {
            const float4 v = src[step * dstride];
            const float2 x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);  // (a, b) of the columns
            const float s0 = v.x + v.y, s1 = v.z + v.w;                           // (a + b) of each column
            const float2 ss0 = make_float2(s0, s0), ss1 = make_float2(s1, s1);
            const float4* rec = tr + step * REC;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              const float4 w = rec[q];
              k12a[2 * q] = __ffma2_rn(make_float2(w.x, w.y), x0, k12a[2 * q]);  // (K2, K3), column cp
              k12b[2 * q] = __ffma2_rn(make_float2(w.x, w.y), x1, k12b[2 * q]);  // (K2, K3), column cp + 1
              if (2 * q + 1 < LG) {
                k12a[2 * q + 1] = __ffma2_rn(make_float2(w.z, w.w), x0, k12a[2 * q + 1]);
                k12b[2 * q + 1] = __ffma2_rn(make_float2(w.z, w.w), x1, k12b[2 * q + 1]);
              }
            }
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              const float4 cv = rec[NP + q];
              k1a[2 * q] = __ffma2_rn(make_float2(cv.x, cv.y), ss0, k1a[2 * q]);  // K1 of loops 4q, 4q + 1
              k1b[2 * q] = __ffma2_rn(make_float2(cv.x, cv.y), ss1, k1b[2 * q]);
              if (2 * q + 1 < NP) {
                k1a[2 * q + 1] = __ffma2_rn(make_float2(cv.z, cv.w), ss0, k1a[2 * q + 1]);
                k1b[2 * q + 1] = __ffma2_rn(make_float2(cv.z, cv.w), ss1, k1b[2 * q + 1]);
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0 && i + ring < total) {
        __threadfence_block();  // this warp's reads of the slot are done before it is counted
        if (atomicAdd(released + slot, 1) == kWarps - 1) {
          released[slot] = 0;
          if (ok) issue(i + ring);
        }
      }
      if (++slot == ring) {
        slot = 0;
        parity ^= 1u;
      }
    }

    // ---- epilogue: column weights, shuffle over lane bits that keep (class, residue), then across warps
    const float2* cw_g = a.colw + static_cast<int64_t>(cc) * LG * W;
    const int lch = CHUNK ? a.lch : LG;  // loops per pass (one pass unless the partials would not fit)
    for (int lc0 = 0; lc0 < LG; lc0 += lch) {
#pragma unroll
    for (int l = 0; l < LG; ++l) {
      if (CHUNK && (l < lc0 || l >= lc0 + lch)) continue;  // another pass's loop (warp-uniform)
      const float2 pa = k12a[l], pb = k12b[l];
      const float c1a = (l & 1) ? k1a[l >> 1].y : k1a[l >> 1].x;  // K1 of loop l, column cp
      const float c1b = (l & 1) ? k1b[l >> 1].y : k1b[l >> 1].x;  // and column cp + 1
      float2 v0 = make_float2(c1a - pa.y, c1a + pa.x);  // (K1 - K3, K1 + K2)
      float2 v1 = make_float2(c1b - pb.y, c1b + pb.x);
      const float2 w0 = smem_colw ? colw[l * W + cp] : __ldg(cw_g + l * W + cp);
      const float2 w1 = smem_colw ? colw[l * W + cp + 1] : __ldg(cw_g + l * W + cp + 1);
      v0 = (ok && active) ? cmul(w0, v0) : make_float2(0.f, 0.f);
      v1 = (ok && active) ? cmul(w1, v1) : make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        if ((rmask >> b) & 1u) {
          v0.x += __shfl_xor_sync(0xffffffffu, v0.x, 1 << b);
          v0.y += __shfl_xor_sync(0xffffffffu, v0.y, 1 << b);
          v1.x += __shfl_xor_sync(0xffffffffu, v1.x, 1 << b);
          v1.y += __shfl_xor_sync(0xffffffffu, v1.y, 1 << b);
        }
      }
      if (leader) {
        const int sl = (warp * nl + lj) * 2;
        red[sl * lch + (l - lc0)] = v0;
        red[(sl + 1) * lch + (l - lc0)] = v1;
      }
    }
    __syncthreads();
    const int nlc = LG - lc0 < lch ? LG - lc0 : lch;
    for (int o = tid; o < nlc * keys; o += kThreads) {
      const int lo = o / keys;
      const int l = lc0 + lo;
      const int key = o - lo * keys;
      const int x = key % X;
      const int cls = cls0 + key / X;
      float2 sum = make_float2(0.f, 0.f);
      for (int k = 0; k < per; ++k) {
        const float2 v = red[static_cast<int>(a.slots[key * per + k]) * lch + lo];
        sum.x += v.x;
        sum.y += v.y;
      }
      if (fs.direct) {
        // bucket j = sigma^{-1} x mod B per dimension (paper order)
        int64_t j = 0;
        int cres = cls;
        int xo[kMaxDim];
#pragma unroll
        for (int d = kMaxDim - 1; d >= 0; --d) {
          xo[d] = 0;
          if (d < fs.d_in) {
            xo[d] = cres & static_cast<int>(g.b[d] - 1);
            cres >>= g.log_b[d];
          }
        }
#pragma unroll
        for (int d = 0; d < kMaxDim; ++d) {
          if (d < g.ndim) {
            const int xd = d < fs.d_in ? xo[d] : static_cast<int>(a.xdig[x * 4 + (d - fs.d_in)]);
            const int jd = (a.sinvb[l * kMaxDim + d] * xd) & static_cast<int>(g.b[d] - 1);
            j += static_cast<int64_t>(jd) << g.b_shift[d];
          }
        }
        folded[static_cast<int64_t>(a.loop0 + l) * g.total_b + j] = sum;
      } else {
        const int ch = rc * fs.col_chunks + cc;
        a.partial[((static_cast<int64_t>(l) * fs.classes + cls) * chunks + ch) * X + x] = sum;
      }
    }
    __syncthreads();  // the partials are read before the next pass or unit writes them
    }
  }
}

struct ReduceArgs {
  Geometry g;
  FoldSchedule fs;
  DeviceTables t;
  int loop0, lg;
  const float2* partial;
  float2* folded;
};

__global__ void fold_reduce_kernel(const ReduceArgs a) {
  const Geometry& g = a.g;
  const FoldSchedule& fs = a.fs;
  const int64_t total = static_cast<int64_t>(a.lg) * fs.classes * fs.xcount;
  const int chunks = fs.row_chunks * fs.col_chunks;
  for (int64_t o = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; o < total;
       o += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(o % fs.xcount);
    const int cls = static_cast<int>((o / fs.xcount) % fs.classes);
    const int l = static_cast<int>(o / (static_cast<int64_t>(fs.xcount) * fs.classes));
    const float2* p = a.partial + ((static_cast<int64_t>(l) * fs.classes + cls) * chunks) * fs.xcount + x;
    float2 sum = make_float2(0.f, 0.f);
    for (int ch = 0; ch < chunks; ++ch) {
      const float2 v = p[static_cast<int64_t>(ch) * fs.xcount];
      sum.x += v.x;
      sum.y += v.y;
    }
    const int lg = a.loop0 + l;
    int c = cls;
    int xo[kMaxDim];
#pragma unroll
    for (int e = kMaxDim - 1; e >= 0; --e) {
      xo[e] = 0;
      if (e < fs.d_in) {
        xo[e] = c & static_cast<int>(g.b[e] - 1);
        c >>= g.log_b[e];
      }
    }
    int64_t j = 0;
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d) {
      if (d < g.ndim) {
        const int xd = d < fs.d_in ? xo[d] : a.t.x_digits[x * 4 + (d - fs.d_in)];
        const int jd = (a.t.sigma_inv_b[lg * g.ndim + d] * xd) & static_cast<int>(g.b[d] - 1);
        j += static_cast<int64_t>(jd) << g.b_shift[d];
      }
    }
    a.folded[static_cast<int64_t>(lg) * g.total_b + j] = sum;
  }
}

template <int LG, bool CHUNK, bool FULL>
cudaError_t launch_fold_shape(const FoldArgs& args, int smem, cudaStream_t stream) {
  int resident = 0;
  const cudaError_t e =
      device_resident_ctas(reinterpret_cast<const void*>(fold_kernel<LG, CHUNK, FULL>), kThreads, smem, &resident);
  if (e != cudaSuccess) return e;
  const int units = args.fs.groups * args.fs.row_chunks * args.fs.col_chunks * args.nframes;
  const int grid = units < resident ? units : resident;
  return launch_chained(fold_kernel<LG, CHUNK, FULL>, dim3(grid), dim3(kThreads), static_cast<size_t>(smem), stream, args);
}

// The constant-stride form up to 12 loops per group: there it is 4-8% faster (radar cube, the
// batched shapes, the 4-D cube at 12 loops); at 16 loops it was slower (4-D cube 2.33 against
// 1.90 ms, 4096 x 4096 114 against 108 us) or equal.
constexpr int kFullMaxLoops = 12;

template <int LG, bool CHUNK>
cudaError_t launch_fold_lg(const FoldArgs& args, int smem, cudaStream_t stream) {
  if constexpr (LG <= kFullMaxLoops) {
    const FoldSchedule& fs = args.fs;
    if (fs.cps * fs.crow * fs.width == kStepElems && fold_stage_steps(fs) == kStepsPerStage)
      return launch_fold_shape<LG, CHUNK, true>(args, smem, stream);
  }
  return launch_fold_shape<LG, CHUNK, false>(args, smem, stream);
}

// One CTA waits, through the fold's bounded barrier wait, on a barrier that nothing
// arrives on: the wait gives up after limit_ns and reports it the way the fold does (the CTA's
// abort flag, then *err = 1).  No copy is in flight and no tensor memory is held.
__global__ void wait_selftest_kernel(int* err, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();
  mbar_wait(&bar, 0u, &abort_flag, err, limit_ns);
}

}  // namespace

cudaError_t launch_wait_selftest(int* err, uint64_t limit_ns, cudaStream_t stream) {
  wait_selftest_kernel<<<1, 32, 0, stream>>>(err, limit_ns);
  return cudaGetLastError();
}

int fold_smem_bytes(const Geometry& g, const FoldSchedule& fs, int lg) {
  (void)g;
  int a, b, c, d, e;
  int f;
  return fold_layout(fs, lg, &a, &b, &c, &d, &e, &f);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  // looked up once; the initialisation of a function-local static is thread-safe
  static const EncodeTiledFn fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    EncodeTiledFn f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess && ptr)
      f = reinterpret_cast<EncodeTiledFn>(ptr);
    cudaGetLastError();
    return f;
  }();
  return fn;
}

// Tensor map of the fold's row boxes: dim 0 = a row's complex elements (8-byte units),
// then for each row dimension d (last first) its residue x_d (size B_d) and its alias
// index m_d (size M_d), so a class's run of local rows is one box.  Returns the rank
// (3 or 5), or 0 when the geometry needs per-row 1-D copies instead.
int encode_fold_map(const Geometry& g, const FoldSchedule& fs, const float2* cube, CUtensorMap* map) {
  if (fs.d_in < 1 || fs.d_in > 2 || fs.width > 256) return 0;
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return 0;
  const int nrows = fold_stage_steps(fs) * fs.crow;  // rows per class per stage
  if (fs.cps > 256) return 0;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  dims[0] = static_cast<cuuint64_t>(fs.row_len);
  box[0] = static_cast<cuuint32_t>(fs.width);
  int rank = 1;
  int64_t sd = fs.row_len;  // element stride of s_d
  int left = nrows;
  for (int d = fs.d_in - 1; d >= 0; --d) {
    const int64_t md = g.m[d];
    const int bm = static_cast<int>(left < md ? left : md);
    if (bm > 256) return 0;
    dims[rank] = static_cast<cuuint64_t>(g.b[d]);
    strides[rank - 1] = static_cast<cuuint64_t>(sd * 8);
    box[rank] = d == fs.d_in - 1 ? static_cast<cuuint32_t>(fs.cps) : 1u;  // the C classes of a unit
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

cudaError_t launch_fold_frames(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t,
                               const float2* const* cubes, int nframes, int64_t folded_stride, int loop0, int lg,
                               float2* folded, float2* partial, int* err, int* copy_mode, cudaStream_t stream,
                               const FoldClear& clear) {
  if (nframes < 1 || nframes > kMaxFrames || (nframes > 1 && !fs.direct)) return cudaErrorInvalidValue;
  thread_local FoldArgs args;  // large (parameter tables); filled, then copied by the launch
  args.tensor_rank = encode_fold_map(g, fs, cubes[0], &args.tmap[0]);
  for (int f = 1; f < nframes; ++f)
    if (encode_fold_map(g, fs, cubes[f], &args.tmap[f]) != args.tensor_rank) return cudaErrorInvalidValue;
  if (copy_mode) *copy_mode = args.tensor_rank;
  for (int f = 0; f < kMaxFrames; ++f) args.cube[f] = cubes[f < nframes ? f : 0];
  args.nframes = nframes;
  args.folded_stride = folded_stride;
  args.clear = clear;
  args.g = g;
  args.fs = fs;
  args.loop0 = loop0;
  args.lg = lg;
  int lw = 0;
  while ((1 << lw) < fs.width) ++lw;
  args.log_width = lw;
  args.folded = folded;
  args.partial = partial;
  args.err = err;
  if (t.ftable_group < 1 || loop0 % t.ftable_group != 0 || lg > t.ftable_group) return cudaErrorInvalidValue;
  args.table = t.ftable + static_cast<int64_t>(loop0 / t.ftable_group) * t.ftable_group_f4;
  args.colw = t.fcolw + static_cast<int64_t>(loop0) * fs.col_chunks * fs.width;
  args.smem_colw = colw_staged(fs, lg) ? 1 : 0;
  for (int l = 0; l < kMaxLoopGroup; ++l)
    for (int d = 0; d < kMaxDim; ++d)
      args.sinvb[l * kMaxDim + d] = (l < lg && d < g.ndim) ? t.h_sinvb[(loop0 + l) * g.ndim + d] : 0;
  const int nslots = fs.slots_per_x * fs.cps * fs.xcount;  // one list per (class in step, residue)
  for (int i = 0; i < nslots && i < 512; ++i) args.slots[i] = t.h_slots[i];
  for (int i = 0; i < fs.xcount * 4 && i < 2048; ++i) args.xdig[i] = t.h_xdig[i];
  const int smem = fold_layout(fs, lg, &args.ring, &args.slot_bytes, &args.colw_off, &args.red_off, &args.bar_off,
                               &args.lch);
  {
    const int chunks = fs.row_chunks * fs.col_chunks;
    args.dv.nst = divisor(stage_shape(fs, lg).nst);
    args.dv.upf = divisor(fs.groups * chunks);
    args.dv.cc = divisor(fs.col_chunks);
    args.dv.rc = divisor(fs.row_chunks);
    args.dv.ch = divisor(chunks);
    args.dv.ring = divisor(args.ring);
  }
  // the epilogue partials of at most 6 loops always fit: multi-pass kernels only above that
  const bool chunk = args.lch < lg;
  switch (lg) {
    case 1: return launch_fold_lg<1, false>(args, smem, stream);
    case 2: return launch_fold_lg<2, false>(args, smem, stream);
    case 3: return launch_fold_lg<3, false>(args, smem, stream);
    case 4: return launch_fold_lg<4, false>(args, smem, stream);
    case 5: return launch_fold_lg<5, false>(args, smem, stream);
    case 6: return launch_fold_lg<6, false>(args, smem, stream);
    case 7: return chunk ? launch_fold_lg<7, true>(args, smem, stream) : launch_fold_lg<7, false>(args, smem, stream);
    case 8: return chunk ? launch_fold_lg<8, true>(args, smem, stream) : launch_fold_lg<8, false>(args, smem, stream);
    case 9: return chunk ? launch_fold_lg<9, true>(args, smem, stream) : launch_fold_lg<9, false>(args, smem, stream);
    case 10: return chunk ? launch_fold_lg<10, true>(args, smem, stream) : launch_fold_lg<10, false>(args, smem, stream);
    case 11: return chunk ? launch_fold_lg<11, true>(args, smem, stream) : launch_fold_lg<11, false>(args, smem, stream);
    case 12: return chunk ? launch_fold_lg<12, true>(args, smem, stream) : launch_fold_lg<12, false>(args, smem, stream);
    case 13: return chunk ? launch_fold_lg<13, true>(args, smem, stream) : launch_fold_lg<13, false>(args, smem, stream);
    case 14: return chunk ? launch_fold_lg<14, true>(args, smem, stream) : launch_fold_lg<14, false>(args, smem, stream);
    case 15: return chunk ? launch_fold_lg<15, true>(args, smem, stream) : launch_fold_lg<15, false>(args, smem, stream);
    case 16: return chunk ? launch_fold_lg<16, true>(args, smem, stream) : launch_fold_lg<16, false>(args, smem, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fold(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t,
                        const float2* cube, int loop0, int lg, float2* folded, float2* partial, int* err,
                        int* copy_mode, cudaStream_t stream, const FoldClear& clear) {
  return launch_fold_frames(g, fs, t, &cube, 1, 0, loop0, lg, folded, partial, err, copy_mode, stream, clear);
}

cudaError_t launch_fold_reduce(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t,
                               int loop0, int lg, const float2* partial, float2* folded,
                               cudaStream_t stream) {
  ReduceArgs args;
  args.g = g;
  args.fs = fs;
  args.t = t;
  args.loop0 = loop0;
  args.lg = lg;
  args.partial = partial;
  args.folded = folded;
  const int64_t total = static_cast<int64_t>(lg) * fs.classes * fs.xcount;
  int blocks = static_cast<int>((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  fold_reduce_kernel<<<blocks, 256, 0, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace rsft
