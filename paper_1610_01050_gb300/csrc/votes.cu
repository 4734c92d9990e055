// vote_scatter, stage2_compact and median_estimate.
//
// vote_scatter: reverse mapping and accumulation of Algorithm 1.  Every
// detected bucket k of loop l expands to its candidate set
// R(k, sigma_l^{-1}) = {sigma^{-1} (k_d M_d + u_d) mod N_d} (Def. 4, Cartesian
// product over dimensions, §III-C.4) and each candidate gets one vote
// (eq. (a_i)).  Votes are 8-bit counters packed four to a 32-bit word and
// incremented with atomic adds; a location gets at most one vote per loop
// (distinctiveness, Prop. 4), so with L <= 255 no byte carries into its
// neighbour.  Lanes of a warp whose candidates share a word are combined
// first (match + ballot), so each word gets one atomic per warp step.
//
// stage2_compact: o = {i : votes[i] > mu} in ascending order (second-stage
// detection, §III-C.5), with the votes cleared for the next call.  A count
// pass, a single-CTA scan of the per-segment counts and an ordered write pass.
//
// median_estimate: for each located i and every loop l, the bucket value
// f-hat_l[M(i, sigma_l)] (Def. 3) divided by the flat-window gain at the
// tone's pass-band offset and by the pre-window's DC gain; the estimate is
// the median of the real parts plus j times the median of the imaginary
// parts over loops (the estimation paragraph of §III).
#include <mutex>
#include <string>

#include "device.cuh"
#include "rsft.h"
#include "tma.cuh"

namespace rsft {
namespace {

constexpr int kSegThreads = 256;
constexpr int kSegIters = 4;
constexpr int64_t kSegBytes = int64_t(kSegThreads) * 16 * kSegIters;  // 16 KiB per segment

struct VoteArgs {
  Geometry g;
  DeviceTables t;
  const uint32_t* det_bits;
  int64_t words_b;
  uint32_t* votes;
};

// One warp per detection word; lanes share out the candidates of each set bit.
__global__ void __launch_bounds__(256) vote_scatter_kernel(const VoteArgs a) {
  const Geometry& g = a.g;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  const int64_t words = static_cast<int64_t>(g.loops) * a.words_b;
  int64_t mtot = 1;
  for (int d = 0; d < g.ndim; ++d) mtot *= g.m[d];
  for (int64_t wi = warp; wi < words; wi += nwarps) {
    uint32_t bits = __ldg(a.det_bits + wi);
    if (!bits) continue;
    const int l = static_cast<int>(wi / a.words_b);
    const int64_t kbase = (wi - static_cast<int64_t>(l) * a.words_b) * 32;
    uint32_t sinv[kMaxDim];
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d) sinv[d] = d < g.ndim ? static_cast<uint32_t>(a.t.sigma_inv[l * g.ndim + d]) : 0u;
    while (bits) {
      const int bpos = __ffs(bits) - 1;
      bits &= bits - 1;
      const int64_t k = kbase + bpos;
      uint32_t kd[kMaxDim];
#pragma unroll
      for (int d = 0; d < kMaxDim; ++d)
        kd[d] = d < g.ndim ? static_cast<uint32_t>((k >> g.b_shift[d]) & (g.b[d] - 1)) : 0u;
      for (int64_t u0 = 0; u0 < mtot; u0 += 32) {
        const int64_t u = u0 + lane;
        const bool valid = u < mtot;
        int64_t i = 0;
        if (valid) {
          int64_t rem = u;
#pragma unroll
          for (int d = kMaxDim - 1; d >= 0; --d) {
            if (d < g.ndim) {
              const uint32_t ud = static_cast<uint32_t>(rem & (g.m[d] - 1));
              rem >>= g.log_m[d];
              // sigma^{-1} (k_d M_d + u_d) mod N_d in 32-bit arithmetic (N_d divides 2^32)
              const uint32_t id = (sinv[d] * ((kd[d] << g.log_m[d]) + ud)) & static_cast<uint32_t>(g.n[d] - 1);
              i += static_cast<int64_t>(id) << g.n_shift[d];
            }
          }
        }
        const unsigned active = __ballot_sync(0xffffffffu, valid);
        if (!valid) continue;
        const unsigned long long word = static_cast<unsigned long long>(i >> 2);
        const int byte = static_cast<int>(i & 3);
        const unsigned peers = __match_any_sync(active, word);
        uint32_t inc = 0;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const unsigned has = __ballot_sync(active, byte == bb) & peers;
          if (has) inc |= 1u << (8 * bb);
        }
        if (lane == __ffs(peers) - 1) atomicAdd(a.votes + word, inc);
      }
    }
  }
}

__device__ __forceinline__ int count_gt(uint32_t w, uint32_t mu4) {
  // bytes of w greater than mu (unsigned per-byte compare)
  return __popc(__vcmpgtu4(w, mu4)) >> 3;
}

__global__ void __launch_bounds__(kSegThreads) stage2_count_kernel(const uint4* votes, int64_t segments,
                                                                   uint32_t mu4, uint32_t* seg_count) {
  __shared__ int warp_sum[kSegThreads / 32];
  for (int64_t seg = blockIdx.x; seg < segments; seg += gridDim.x) {
    int c = 0;
#pragma unroll
    for (int it = 0; it < kSegIters; ++it) {
      const uint4 v = votes[(seg * kSegIters + it) * kSegThreads + threadIdx.x];
      if (v.x | v.y | v.z | v.w)
        c += count_gt(v.x, mu4) + count_gt(v.y, mu4) + count_gt(v.z, mu4) + count_gt(v.w, mu4);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int w = 0; w < kSegThreads / 32; ++w) tot += warp_sum[w];
      seg_count[seg] = static_cast<uint32_t>(tot);
    }
    __syncthreads();
  }
}

// Single CTA: exclusive scan of the segment counts; offset[segments] = total.
__global__ void __launch_bounds__(1024) stage2_scan_kernel(const uint32_t* seg_count, int64_t segments,
                                                           uint64_t* seg_offset, int64_t* d_count) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < segments; base += 1024) {
    const int64_t i = base + threadIdx.x;
    unsigned long long v = i < segments ? seg_count[i] : 0ull;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      unsigned long long t = warp_tot[lane];
      unsigned long long ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      warp_tot[lane] = ti - t;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    const unsigned long long excl = carry + warp_tot[wid] + incl - v;
    if (i < segments) seg_offset[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    seg_offset[segments] = carry;
    *d_count = static_cast<int64_t>(carry);
  }
}

__global__ void __launch_bounds__(kSegThreads) stage2_write_kernel(
    uint4* votes, int64_t segments, uint32_t mu, uint32_t mu4, const uint64_t* seg_offset,
    uint64_t* located, uint8_t* located_votes, uint8_t* votes_out, int64_t total_n, int64_t capacity) {
  __shared__ int warp_excl[kSegThreads / 32];
  __shared__ int block_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t seg = blockIdx.x; seg < segments; seg += gridDim.x) {
    uint64_t pos = seg_offset[seg];
#pragma unroll 1
    for (int it = 0; it < kSegIters; ++it) {
      const int64_t vi = (seg * kSegIters + it) * kSegThreads + threadIdx.x;
      const uint4 v = votes[vi];
      const bool any = (v.x | v.y | v.z | v.w) != 0u;
      int c = any ? count_gt(v.x, mu4) + count_gt(v.y, mu4) + count_gt(v.z, mu4) + count_gt(v.w, mu4) : 0;
      int incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) warp_excl[wid] = incl;
      __syncthreads();
      if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kSegThreads / 32; ++w) {
          const int t = warp_excl[w];
          warp_excl[w] = run;
          run += t;
        }
        block_tot = run;
      }
      __syncthreads();
      uint64_t out = pos + static_cast<uint64_t>(warp_excl[wid] + incl - c);
      const int64_t byte0 = vi * 16;
      if (c) {
        const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            const uint32_t cnt = (wv[q] >> (8 * bb)) & 0xffu;
            if (cnt > mu) {
              if (out < static_cast<uint64_t>(capacity)) {
                located[out] = static_cast<uint64_t>(byte0 + q * 4 + bb);
                if (located_votes) located_votes[out] = static_cast<uint8_t>(cnt);
              }
              ++out;
            }
          }
        }
      }
      if (any) {
        if (votes_out) {
          if (byte0 + 16 <= total_n) {
            *reinterpret_cast<uint4*>(votes_out + byte0) = v;
          } else {
            const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
            for (int bb = 0; bb < 16 && byte0 + bb < total_n; ++bb)
              votes_out[byte0 + bb] = static_cast<uint8_t>((wv[bb >> 2] >> (8 * (bb & 3))) & 0xffu);
          }
        }
        votes[vi] = make_uint4(0u, 0u, 0u, 0u);
      } else if (votes_out) {
        if (byte0 + 16 <= total_n) {
          *reinterpret_cast<uint4*>(votes_out + byte0) = make_uint4(0u, 0u, 0u, 0u);
        } else {
          for (int bb = 0; bb < 16 && byte0 + bb < total_n; ++bb) votes_out[byte0 + bb] = 0;
        }
      }
      pos += static_cast<uint64_t>(block_tot);
      __syncthreads();
    }
  }
}

struct MedianArgs {
  Geometry g;
  DeviceTables t;
  const float2* spectrum;
  const uint64_t* located;
  const int64_t* d_count;
  int64_t capacity;
  float2* amp;
};

// The median kernels' pointers of frame blockIdx.y (frames one after another: [frame][L][B]
// spectra, capacity located entries and one count per frame).
struct MedianFrame {
  const float2* spectrum;
  const uint64_t* located;
  const int64_t* d_count;
  float2* amp;
};

__device__ __forceinline__ MedianFrame median_frame(const MedianArgs& a) {
  const int64_t f = blockIdx.y;
  MedianFrame m;
  m.spectrum = a.spectrum + f * a.g.loops * a.g.total_b;
  m.located = a.located + f * a.capacity;
  m.d_count = a.d_count + f;
  m.amp = a.amp + f * a.capacity;
  return m;
}

constexpr int kMedianWarps = 4;

// One warp per located index; per-loop values in shared memory, median by rank.
__global__ void __launch_bounds__(kMedianWarps * 32) median_kernel(const MedianArgs a) {
  chain_wait();
  chain_release();
  const MedianFrame mf = median_frame(a);
  __shared__ float vre[kMedianWarps][256];
  __shared__ float vim[kMedianWarps][256];
  __shared__ float sel[kMedianWarps][4];
  const Geometry& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t count = *mf.d_count;
  if (count > a.capacity) count = a.capacity;
  const int L = g.loops;
  const int lo_rank = (L - 1) / 2, hi_rank = L / 2;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * kMedianWarps + wid; q < count;
       q += static_cast<int64_t>(gridDim.x) * kMedianWarps) {
    const uint64_t i = mf.located[q];
    uint32_t id[kMaxDim];
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d)
      id[d] = d < g.ndim ? static_cast<uint32_t>((i >> g.n_shift[d]) & static_cast<uint64_t>(g.n[d] - 1)) : 0u;
    for (int l = lane; l < L; l += 32) {
      int64_t k = 0;
      float2 val = make_float2(1.f, 0.f);
#pragma unroll
      for (int d = 0; d < kMaxDim; ++d) {
        if (d < g.ndim) {
          const uint32_t p = (static_cast<uint32_t>(a.t.sigma[l * g.ndim + d]) * id[d]) &
                             static_cast<uint32_t>(g.n[d] - 1);  // [sigma i]_N
          const uint32_t kd = p >> g.log_m[d];                  // M(i, sigma), Def. 3
          const uint32_t v = p & static_cast<uint32_t>(g.m[d] - 1);
          k += static_cast<int64_t>(kd) << g.b_shift[d];
          const float2 gi = __ldg(a.t.ginv[d] + v);
          val = make_float2(val.x * gi.x - val.y * gi.y, val.x * gi.y + val.y * gi.x);
        }
      }
      const float2 f = mf.spectrum[static_cast<int64_t>(l) * g.total_b + k];
      vre[wid][l] = f.x * val.x - f.y * val.y;
      vim[wid][l] = f.x * val.y + f.y * val.x;
    }
    __syncwarp();
    for (int l = lane; l < L; l += 32) {
      const float xr = vre[wid][l], xi = vim[wid][l];
      int rr = 0, ri = 0;
      for (int m2 = 0; m2 < L; ++m2) {
        const float yr = vre[wid][m2], yi = vim[wid][m2];
        rr += (yr < xr) || (yr == xr && m2 < l);
        ri += (yi < xi) || (yi == xi && m2 < l);
      }
      if (rr == lo_rank) sel[wid][0] = xr;
      if (rr == hi_rank) sel[wid][1] = xr;
      if (ri == lo_rank) sel[wid][2] = xi;
      if (ri == hi_rank) sel[wid][3] = xi;
    }
    __syncwarp();
    if (lane == 0) mf.amp[q] = make_float2(0.5f * (sel[wid][0] + sel[wid][1]), 0.5f * (sel[wid][2] + sel[wid][3]));
    __syncwarp();
  }
}

// Loops of G lanes (L <= G): 32 / G located indices per warp, the per-loop
// values stay in registers and the ranks come from shuffles within the group.
template <int G>
__global__ void __launch_bounds__(kMedianWarps * 32) median_group_kernel(const MedianArgs a) {
  chain_wait();
  chain_release();
  const MedianFrame mf = median_frame(a);
  const Geometry& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int sub = lane / G, l = lane % G;
  constexpr int kPerWarp = 32 / G;
  int64_t count = *mf.d_count;
  if (count > a.capacity) count = a.capacity;
  const int L = g.loops;
  const int lo_rank = (L - 1) / 2, hi_rank = L / 2;
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (sub * G);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * kMedianWarps * kPerWarp;
  for (int64_t base = (static_cast<int64_t>(blockIdx.x) * kMedianWarps + wid) * kPerWarp; base < count;
       base += stride) {
    const int64_t q = base + sub;
    const bool active = q < count && l < L;
    float xr = 0.f, xi = 0.f;
    if (active) {
      const uint64_t i = mf.located[q];
      int64_t k = 0;
      float2 val = make_float2(1.f, 0.f);
#pragma unroll
      for (int d = 0; d < kMaxDim; ++d) {
        if (d < g.ndim) {
          const uint32_t id = static_cast<uint32_t>((i >> g.n_shift[d]) & static_cast<uint64_t>(g.n[d] - 1));
          const uint32_t p = (static_cast<uint32_t>(a.t.sigma[l * g.ndim + d]) * id) &
                             static_cast<uint32_t>(g.n[d] - 1);  // [sigma i]_N
          const uint32_t kd = p >> g.log_m[d];                  // M(i, sigma), Def. 3
          const uint32_t v = p & static_cast<uint32_t>(g.m[d] - 1);
          k += static_cast<int64_t>(kd) << g.b_shift[d];
          const float2 gi = __ldg(a.t.ginv[d] + v);
          val = make_float2(val.x * gi.x - val.y * gi.y, val.x * gi.y + val.y * gi.x);
        }
      }
      const float2 f = mf.spectrum[static_cast<int64_t>(l) * g.total_b + k];
      xr = f.x * val.x - f.y * val.y;
      xi = f.x * val.y + f.y * val.x;
    }
    int rr = 0, ri = 0;
    for (int m2 = 0; m2 < L; ++m2) {
      const float yr = __shfl_sync(0xffffffffu, xr, m2, G);
      const float yi = __shfl_sync(0xffffffffu, xi, m2, G);
      rr += (yr < xr) || (yr == xr && m2 < l);
      ri += (yi < xi) || (yi == xi && m2 < l);
    }
    // ranks are a permutation of [0, L): exactly one lane of an active group holds each
    const unsigned b0 = __ballot_sync(0xffffffffu, active && rr == lo_rank) & gmask;
    const unsigned b1 = __ballot_sync(0xffffffffu, active && rr == hi_rank) & gmask;
    const unsigned b2 = __ballot_sync(0xffffffffu, active && ri == lo_rank) & gmask;
    const unsigned b3 = __ballot_sync(0xffffffffu, active && ri == hi_rank) & gmask;
    const float r0 = __shfl_sync(0xffffffffu, xr, b0 ? __ffs(b0) - 1 : lane);
    const float r1 = __shfl_sync(0xffffffffu, xr, b1 ? __ffs(b1) - 1 : lane);
    const float i0 = __shfl_sync(0xffffffffu, xi, b2 ? __ffs(b2) - 1 : lane);
    const float i1 = __shfl_sync(0xffffffffu, xi, b3 ? __ffs(b3) - 1 : lane);
    if (active && l == 0) mf.amp[q] = make_float2(0.5f * (r0 + r1), 0.5f * (i0 + i1));
  }
}

// ---------------------------------------------------------------------------
// vote_rows: the reverse mapping and accumulation of Algorithm 1 and the
// second-stage detection, organised by output rows instead of by detected
// buckets.  A location i gets one vote from loop l iff bucket M(i, sigma_l)
// was detected (Def. 3 and Prop. 3: i is in R(j, sigma^{-1}) iff j = M(i,
// sigma)), so the votes of an output row (the trailing dimensions [d_v, D) at
// fixed leading indices) come from one plane of B_in buckets per loop.  A lane
// first counts, per row, the loops whose plane holds any detection; a row with
// at most mu such loops cannot pass the second stage and is skipped.  For the
// remaining rows the warp expands the detected buckets of each loop into their
// candidates (Def. 4) and counts votes in shared memory (candidates of one
// loop are distinct, Prop. 4, so a loop's increments never collide), then
// emits {i : votes > mu} in ascending order.  Pass 0 counts the hits of each
// warp, a scan turns them into offsets, pass 1 repeats the work and writes.
struct RowArgs {
  Geometry g;
  DeviceTables t;
  int* err;                 // set when a barrier wait gives up
  const uint32_t* det_bits;
  int64_t words_b;
  int d_v;
  int64_t n_in;
  int b_in;
  int m_in;
  int64_t rows;
  int rows_per_warp;
  int64_t warps;
  int mu;
  uint32_t* warp_count;
  const uint64_t* warp_offset;
  uint64_t* located;
  uint8_t* located_votes;
  uint8_t* votes_out;
  int64_t capacity;
  int64_t* d_count;         // small rows: the total located count (written by the emit kernel)
  ulonglong2* row_list;     // small rows, per warp [rows_per_warp]: (row, its votes > mu mask) of emitting rows
  uint32_t* warp_rows;      // small rows: [warps] entries in the warp's row list
  int64_t frame_bits;       // small rows, frames along blockIdx.y: detection words between frames (multiple of 4)
};

// The small-row kernels' pointers of frame blockIdx.y: its detection bitmaps, warp counts and
// row lists, located list and count (frame 0 is the arguments themselves).
struct FramePtrs {
  const uint32_t* det_bits;
  uint32_t* warp_count;
  uint32_t* warp_rows;
  ulonglong2* row_list;
  uint64_t* located;
  uint8_t* located_votes;
  int64_t* d_count;
};

__device__ __forceinline__ FramePtrs frame_ptrs(const RowArgs& a) {
  const int64_t f = blockIdx.y;
  FramePtrs p;
  p.det_bits = a.det_bits + f * a.frame_bits;
  p.warp_count = a.warp_count + f * a.warps;
  p.warp_rows = a.warp_rows + f * a.warps;
  p.row_list = a.row_list + f * a.warps * a.rows_per_warp;
  p.located = a.located + f * a.capacity;
  p.located_votes = a.located_votes ? a.located_votes + f * a.capacity : nullptr;
  p.d_count = a.d_count + f;
  return p;
}

constexpr int kRowWarps = 8;
static_assert(kRowWarps % 4 == 0, "the emit kernel reads the warp counts four at a time");

// First bucket index of the B_in-bucket plane that row `row` maps to in loop l.
__device__ __forceinline__ int64_t plane_of(const RowArgs& a, int l, int64_t row) {
  const Geometry& g = a.g;
  int64_t kb = 0, r = row;
#pragma unroll
  for (int d = kMaxDim - 1; d >= 0; --d) {
    if (d < a.d_v) {
      const uint32_t id = static_cast<uint32_t>(r & (g.n[d] - 1));
      r >>= g.log_n[d];
      const uint32_t p = (static_cast<uint32_t>(a.t.sigma[l * g.ndim + d]) * id) & static_cast<uint32_t>(g.n[d] - 1);
      kb += static_cast<int64_t>(p >> g.log_m[d]) << g.b_shift[d];
    }
  }
  return kb;
}

// Detection bits [kb, kb + B_in) of loop l, word w of the plane (one word when B_in <= 32).
// `bits` is the detection bitmap, staged in shared memory when it fits.
__device__ __forceinline__ uint32_t plane_word(const RowArgs& a, const uint32_t* bits, int l, int64_t kb, int w) {
  const uint32_t* b = bits + static_cast<int64_t>(l) * a.words_b;
  if (a.b_in < 32) return (b[kb >> 5] >> (kb & 31)) & ((1u << a.b_in) - 1u);
  return b[(kb >> 5) + w];
}

__device__ __forceinline__ bool plane_any(const RowArgs& a, const uint32_t* bits, int l, int64_t kb) {
  const int words = a.b_in < 32 ? 1 : (a.b_in >> 5);
  for (int w = 0; w < words; ++w)
    if (plane_word(a, bits, l, kb, w)) return true;
  return false;
}

template <int PASS>
__global__ void __launch_bounds__(kRowWarps * 32) vote_rows_kernel(const RowArgs a, int staged) {
  extern __shared__ uint32_t smem_words[];
  const Geometry& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t cwords = (a.n_in + 3) >> 2;
  const int64_t bit_words = static_cast<int64_t>(g.loops) * a.words_b;
  const uint32_t* bits = a.det_bits;
  if (staged) {
    // all L detection bitmaps, copied once per CTA (latency of shared memory instead of L2)
    uint32_t* sb = smem_words + kRowWarps * cwords;
    for (int64_t w = threadIdx.x; w < bit_words; w += kRowWarps * 32) sb[w] = __ldg(a.det_bits + w);
    __syncthreads();
    bits = sb;
  }
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * kRowWarps + wid;
  if (gw >= a.warps) return;  // no block-wide barriers below
  uint32_t* cnt = smem_words + wid * cwords;
  uint8_t* cnt8 = reinterpret_cast<uint8_t*>(cnt);
  for (int64_t w = lane; w < cwords; w += 32) cnt[w] = 0u;
  __syncwarp();
  const int L = g.loops;
  const bool full = PASS == 1 && a.votes_out != nullptr;
  const uint32_t mu4 = static_cast<uint32_t>(a.mu) * 0x01010101u;
  uint64_t pos = PASS == 1 ? a.warp_offset[gw] : 0ull;
  uint32_t hits = 0;
  const int64_t row0 = gw * a.rows_per_warp;
  const int plane_words = a.b_in < 32 ? 1 : (a.b_in >> 5);
  for (int rb = 0; rb < a.rows_per_warp; rb += 32) {
    const int64_t row = row0 + rb + lane;
    const bool valid = rb + lane < a.rows_per_warp && row < a.rows;
    int nz = 0;
    if (valid && !full) {
#pragma unroll 4
      for (int l = 0; l < L; ++l) nz += plane_any(a, bits, l, plane_of(a, l, row)) ? 1 : 0;
    }
    unsigned cand = __ballot_sync(0xffffffffu, valid && (full || nz > a.mu));
    while (cand) {
      const int src = __ffs(cand) - 1;
      cand &= cand - 1;
      const int64_t crow = row0 + rb + src;
      // ---- votes of row crow
      for (int l0 = 0; l0 < L; l0 += 32) {
        const int l = l0 + lane;
        int64_t kb = 0;
        bool live = false;
        if (l < L) {
          kb = plane_of(a, l, crow);
          live = plane_any(a, bits, l, kb);
        }
        unsigned lm = __ballot_sync(0xffffffffu, live);
        while (lm) {
          const int ls = __ffs(lm) - 1;
          lm &= lm - 1;
          const int ll = l0 + ls;
          const int64_t kbl = __shfl_sync(0xffffffffu, kb, ls);
          for (int pw = 0; pw < plane_words; ++pw) {
            uint32_t word = plane_word(a, bits, ll, kbl, pw);
            while (word) {
              const int b = pw * 32 + __ffs(word) - 1;
              word &= word - 1;
              for (int u = lane; u < a.m_in; u += 32) {
                // candidate sigma^{-1} (b_e M_e + u_e) mod N_e per trailing dimension (Def. 4)
                int64_t iin = 0;
                int mshift = 0;
#pragma unroll
                for (int d = kMaxDim - 1; d >= 0; --d) {
                  if (d >= a.d_v && d < g.ndim) {
                    const uint32_t bd = static_cast<uint32_t>(b >> g.b_shift[d]) & static_cast<uint32_t>(g.b[d] - 1);
                    const uint32_t ud = static_cast<uint32_t>(u >> mshift) & static_cast<uint32_t>(g.m[d] - 1);
                    mshift += g.log_m[d];
                    const uint32_t id = (static_cast<uint32_t>(a.t.sigma_inv[ll * g.ndim + d]) * ((bd << g.log_m[d]) + ud)) &
                                        static_cast<uint32_t>(g.n[d] - 1);
                    iin += static_cast<int64_t>(id) << g.n_shift[d];
                  }
                }
                cnt8[iin] = static_cast<uint8_t>(cnt8[iin] + 1);
              }
            }
          }
          __syncwarp();
        }
      }
      // ---- second stage on the row: votes > mu, ascending; clear the counters
      for (int64_t w0 = 0; w0 < cwords; w0 += 32) {
        const int64_t w = w0 + lane;
        const uint32_t v = w < cwords ? cnt[w] : 0u;
        const int h = v ? (__popc(__vcmpgtu4(v, mu4)) >> 3) : 0;
        if (PASS == 0) {
          hits += static_cast<uint32_t>(h);
        } else {
          int incl = h;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const int tot = __shfl_sync(0xffffffffu, incl, 31);
          uint64_t out = pos + static_cast<uint64_t>(incl - h);
          if (h) {
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
              const uint32_t c = (v >> (8 * bb)) & 0xffu;
              if (c > static_cast<uint32_t>(a.mu)) {
                if (out < static_cast<uint64_t>(a.capacity)) {
                  a.located[out] = static_cast<uint64_t>(crow * a.n_in + w * 4 + bb);
                  if (a.located_votes) a.located_votes[out] = static_cast<uint8_t>(c);
                }
                ++out;
              }
            }
          }
          pos += static_cast<uint64_t>(tot);
          if (full && w < cwords) {
            for (int bb = 0; bb < 4 && w * 4 + bb < a.n_in; ++bb)
              a.votes_out[crow * a.n_in + w * 4 + bb] = static_cast<uint8_t>((v >> (8 * bb)) & 0xffu);
          }
        }
        if (v) cnt[w] = 0u;
      }
      __syncwarp();
    }
  }
  if (PASS == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
    if (lane == 0) a.warp_count[gw] = hits;
  }
}

// vote_rows_small: rows of at most 64 locations.  A lane owns a row; the votes
// of its 64 locations are kept as eight 64-bit bit-planes (bit p of every
// location's count), each loop adds the mask of candidates of its detected
// buckets (the OR of the precomputed masks R(b, sigma_l^{-1}) of the row's
// detected inner buckets b, Def. 4) with a ripple carry, and a bit-sliced
// comparison with mu gives the second-stage hits of all 64 locations at once.
// Shared-memory layout of the small-row kernel (byte offsets, all multiples of 16):
// [0, 16) barrier, then the bucket-offset tables, then (staged) the candidate masks
// and the detection bitmaps.  Copy sizes are rounded up to 16 bytes; the plan pads
// the three device arrays to match.
// Shared-memory layout of the small-row kernels (byte offsets, all multiples of 16):
// [0, 16) barrier, the bucket-offset tables (u16), the candidate table, the detection
// bitmaps.  Copy sizes are rounded up to 16 bytes; the plan pads the device arrays.
struct SmallRowLayout {
  uint32_t kb_bytes, cand_bytes, bit_bytes;
  uint32_t kb_off, cand_off, bit_off, total;
};

__host__ __device__ __forceinline__ uint32_t round16(uint64_t v) { return static_cast<uint32_t>((v + 15) & ~15ull); }

// Candidate table: with B_in <= 8 inner buckets, per loop the union of the candidate masks
// of every detection pattern of a plane ([L][2^B_in]); otherwise one mask per bucket.
__host__ __device__ __forceinline__ bool pattern_table(int b_in) { return b_in <= 8; }

// Bucket-offset tables of the row dimensions: per index i_d the offsets of all loops, padded
// to whole 16-byte groups of eight ([N_d][kb_loops_padded(L)] u16 per dimension).
__host__ __device__ __forceinline__ int kb_loops_padded(int loops) { return (loops + 7) & ~7; }

__host__ __device__ inline SmallRowLayout small_row_layout(const Geometry& g, int d_v, int b_in, int64_t words_b) {
  SmallRowLayout s{};
  int64_t kb_words = 0;
  for (int d = 0; d < d_v; ++d) kb_words += static_cast<int64_t>(kb_loops_padded(g.loops)) * g.n[d];
  s.kb_bytes = round16(static_cast<uint64_t>(kb_words) * 2);
  s.cand_bytes = round16(static_cast<uint64_t>(g.loops) * (pattern_table(b_in) ? (1 << b_in) : b_in) * 8);
  s.bit_bytes = round16(static_cast<uint64_t>(g.loops) * words_b * 4);
  s.kb_off = 16;
  s.cand_off = s.kb_off + s.kb_bytes;
  s.bit_off = s.cand_off + s.cand_bytes;
  s.total = s.bit_off + s.bit_bytes;
  return s;
}

// The tables a row count reads (shared memory, or global memory in the emit kernel).
struct RowTables {
  const uint16_t* kb;      // per row dimension d < d_v: [N_d][kb_loops_padded(L)] bucket offset of index i_d
  const uint64_t* cand;    // [L][2^B_in] pattern unions, or [L][B_in] per-bucket masks
  const uint32_t* bits;    // [L][words_b] detection bitmaps
};

// Votes of the n_in locations of output row `row` as bit-planes (bit i of c[p] = bit p of
// the votes of inner location i; NP planes are counted, the rest stay 0): loop l adds one
// vote to every candidate of the detected buckets of the row's plane (Def. 4; candidates
// of one loop are distinct, Prop. 4).  DV = number of row dimensions.
template <int DV, int NP>
__device__ __forceinline__ void count_row(const RowArgs& a, const RowTables& t, int64_t row, uint64_t* c) {
  const Geometry& g = a.g;
  const int L = g.loops;
  const bool wide = a.b_in > 32;
  const uint32_t pat_mask = a.b_in < 32 ? ((1u << a.b_in) - 1u) : 0xffffffffu;
  const bool table = pattern_table(a.b_in);
  const uint16_t* kp[DV > 0 ? DV : 1];
  int kn[DV > 0 ? DV : 1];
  {
    uint64_t r = static_cast<uint64_t>(row);
    int idx[DV > 0 ? DV : 1];
#pragma unroll
    for (int d = DV - 1; d >= 0; --d) {
      idx[d] = static_cast<int>(static_cast<uint32_t>(r) & static_cast<uint32_t>(g.n[d] - 1));
      r >>= g.log_n[d];
    }
    const int Lp = kb_loops_padded(L);
    int off = 0;
#pragma unroll
    for (int d = 0; d < DV; ++d) {
      kp[d] = t.kb + off + idx[d] * Lp;
      kn[d] = 1;
      off += Lp * static_cast<int>(g.n[d]);
    }
  }
#pragma unroll
  for (int p = 0; p < 8; ++p) c[p] = 0ull;
  const uint32_t* bl = t.bits;
  for (int l = 0; l < L; ++l, bl += a.words_b) {
    uint32_t kb = 0u;
#pragma unroll
    for (int d = 0; d < DV; ++d) {
      kb += *kp[d];
      kp[d] += kn[d];
    }
    uint64_t pat = (bl[kb >> 5] >> (kb & 31u)) & pat_mask;
    if (wide) pat |= static_cast<uint64_t>(bl[(kb >> 5) + 1]) << 32;
    if (!pat) continue;
    uint64_t m;
    if (table) {
      m = t.cand[(l << a.b_in) + static_cast<int>(pat)];
    } else {
      m = 0ull;
      const uint64_t* ml = t.cand + static_cast<int64_t>(l) * a.b_in;
      while (pat) {
        m |= ml[__ffsll(static_cast<long long>(pat)) - 1];
        pat &= pat - 1;
      }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const uint64_t tt = c[p] & m;
      c[p] ^= m;
      m = tt;
    }
  }
}

// Loads from the shared-memory window by 32-bit address.  They read tables that no thread
// writes after the kernel's copy barrier; every address they take derives from a base formed
// after that barrier (shared_base), so the compiler cannot move them above it.
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint64_t lds_u64(uint32_t addr) {
  uint64_t v;
  asm("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint32_t shared_base(const void* p) {
  uint32_t v;
  asm volatile("mov.u32 %0, %1;" : "=r"(v) : "r"(smem_u32(p)));
  return v;
}

// count_row on tables staged in shared memory (window addresses of the bucket-offset tables,
// the candidate table and the detection bitmaps): the same counts.  The offsets of eight loops
// come with one 16-byte load per row dimension and are summed two at a time in 32-bit words
// (an offset sum stays below B <= 65536, so the halves never carry into each other); each loop
// then costs one bitmap load and a few integer operations unless its plane holds a detection.
template <int DV, int NP>
__device__ __forceinline__ void count_row_smem(const RowArgs& a, uint32_t s_kb, uint32_t s_cand, uint32_t s_bits,
                                               int64_t row, uint64_t* c) {
  const Geometry& g = a.g;
  const int L = g.loops;
  const uint32_t Lp = static_cast<uint32_t>(kb_loops_padded(L));
  const bool wide = a.b_in > 32;
  const uint32_t pat_mask = a.b_in < 32 ? ((1u << a.b_in) - 1u) : 0xffffffffu;
  const bool table = pattern_table(a.b_in);
  uint32_t ka[DV > 0 ? DV : 1];
  {
    uint64_t r = static_cast<uint64_t>(row);
    uint32_t idx[DV > 0 ? DV : 1];
#pragma unroll
    for (int d = DV - 1; d >= 0; --d) {
      idx[d] = static_cast<uint32_t>(r) & static_cast<uint32_t>(g.n[d] - 1);
      r >>= g.log_n[d];
    }
    uint32_t off = 0;
#pragma unroll
    for (int d = 0; d < DV; ++d) {
      ka[d] = s_kb + 2u * (off + idx[d] * Lp);
      off += static_cast<uint32_t>(g.n[d]) * Lp;
    }
  }
#pragma unroll
  for (int p = 0; p < 8; ++p) c[p] = 0ull;
  const uint32_t wstep = 32u * static_cast<uint32_t>(a.words_b);  // bits of one loop's bitmap
  const uint32_t cstep = 8u * static_cast<uint32_t>(table ? (1 << a.b_in) : a.b_in);
  uint32_t boff = 0u;                                              // first bit of loop l's bitmap
  for (int l0 = 0; l0 < L; l0 += 8) {
    uint32_t kw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int d = 0; d < DV; ++d) {
      uint32_t t0, t1, t2, t3;
      asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(t0), "=r"(t1), "=r"(t2), "=r"(t3) : "r"(ka[d] + 2u * l0));
      kw[0] += t0;
      kw[1] += t1;
      kw[2] += t2;
      kw[3] += t3;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (l0 + j < L) {
        const uint32_t kb = ((kw[j >> 1] >> (16 * (j & 1))) & 0xffffu) + boff;
        const uint32_t wa = s_bits + ((kb >> 5) << 2);
        const uint32_t plo = (lds_u32(wa) >> (kb & 31u)) & pat_mask;
        const uint32_t phi = wide ? lds_u32(wa + 4u) : 0u;
        if (plo | phi) {
          const uint32_t sc = s_cand + static_cast<uint32_t>(l0 + j) * cstep;
          uint64_t m;
          if (table) {
            m = lds_u64(sc + (plo << 3));
          } else {
            m = 0ull;
            uint64_t pat = static_cast<uint64_t>(plo) | (static_cast<uint64_t>(phi) << 32);
            while (pat) {
              m |= lds_u64(sc + (static_cast<uint32_t>(__ffsll(static_cast<long long>(pat)) - 1) << 3));
              pat &= pat - 1;
            }
          }
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const uint64_t tt = c[p] & m;
            c[p] ^= m;
            m = tt;
          }
        }
      }
      boff += wstep;
    }
  }
}

// Locations of the row with votes > mu, bit-sliced (NP counter planes; votes < 2^NP).
template <int NP>
__device__ __forceinline__ uint64_t above_mu(const RowArgs& a, const uint64_t* c) {
  if (a.mu >> NP) return 0ull;  // more votes than NP planes can hold
  uint64_t eq = ~0ull, gt = 0ull;
#pragma unroll
  for (int p = NP - 1; p >= 0; --p) {
    if ((a.mu >> p) & 1) {
      eq &= c[p];
    } else {
      gt |= eq & c[p];
      eq &= ~c[p];
    }
  }
  return gt & (a.n_in >= 64 ? ~0ull : ((1ull << a.n_in) - 1ull));
}

__device__ __forceinline__ uint8_t votes_of(const uint64_t* c, int bit) {
  uint32_t v = 0;
#pragma unroll
  for (int p = 0; p < 8; ++p) v |= static_cast<uint32_t>((c[p] >> bit) & 1ull) << p;
  return static_cast<uint8_t>(v);
}

// Write the located indices (and votes) of one row per lane, in lane order, from `pos`.
__device__ __forceinline__ uint64_t write_rows(const RowArgs& a, const FramePtrs& fp, int lane, int64_t row, uint64_t gt,
                                               const uint64_t* c, uint64_t pos) {
  const int h = __popcll(gt);
  int incl = h;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int tot = __shfl_sync(0xffffffffu, incl, 31);
  uint64_t out = pos + static_cast<uint64_t>(incl - h);
  uint64_t rem = gt;
  while (rem) {
    const int bit = __ffsll(static_cast<long long>(rem)) - 1;
    rem &= rem - 1;
    if (out < static_cast<uint64_t>(a.capacity)) {
      fp.located[out] = static_cast<uint64_t>(row * a.n_in + bit);
      if (fp.located_votes) fp.located_votes[out] = votes_of(c, bit);
    }
    ++out;
  }
  return pos + static_cast<uint64_t>(tot);
}

// Small rows (<= 64 locations), one lane per row with 8 bit-planes of u64 counters.
// PASS 0: count every row, list the rows with votes > mu (row, mask) per warp, count hits.
// PASS 1 (the full vote array only): recount every row, write located indices in order
// from the scanned warp offsets, and every row's votes.
constexpr int kSmallWarps = 16;

template <int PASS, int DV, int NP>
__global__ void __launch_bounds__(kSmallWarps * 32) vote_rows_small_kernel(const RowArgs a) {
  extern __shared__ __align__(16) unsigned char smem_small[];
  const FramePtrs fp = frame_ptrs(a);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const SmallRowLayout lay = small_row_layout(a.g, a.d_v, a.b_in, a.words_b);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_small);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // the plan's offset and candidate tables (written at plan creation) load while the previous
    // kernel of the chain finishes; the detection bitmaps only after it has
    const uint64_t pol = policy_evict_last();
    mbar_arrive_expect_tx(bar, lay.kb_bytes + lay.cand_bytes + lay.bit_bytes);
    if (lay.kb_bytes) bulk_g2s(smem_small + lay.kb_off, a.t.kb16, lay.kb_bytes, bar, pol);  // none when d_v == 0
    bulk_g2s(smem_small + lay.cand_off, a.t.rowmask, lay.cand_bytes, bar, pol);
  }
  chain_wait();
  chain_release();
  if (threadIdx.x == 0) bulk_g2s(smem_small + lay.bit_off, fp.det_bits, lay.bit_bytes, bar, policy_evict_last());
  if (!mbar_wait_bounded(bar, 0u, a.err)) return;  // no block-wide barriers below
  const int64_t gw = static_cast<int64_t>(blockIdx.x) * kSmallWarps + wid;
  if (gw >= a.warps) return;
  const uint32_t sbase = shared_base(smem_small);   // (after the copy barrier)
  const uint32_t s_kb = sbase + lay.kb_off, s_cand = sbase + lay.cand_off, s_bits = sbase + lay.bit_off;
  const int64_t row0 = gw * a.rows_per_warp;
  ulonglong2* list = fp.row_list + row0;
  uint64_t pos = PASS == 1 ? a.warp_offset[gw] : 0ull;
  uint32_t hits = 0, nlist = 0;
  for (int rb = 0; rb < a.rows_per_warp; rb += 32) {
    const int64_t row = row0 + rb + lane;
    const bool valid = rb + lane < a.rows_per_warp && row < a.rows;
    uint64_t c[8];
    uint64_t gt = 0ull;
    if (valid) {
      count_row_smem<DV, NP>(a, s_kb, s_cand, s_bits, row, c);
      gt = above_mu<NP>(a, c);
    }
    if (PASS == 0) {
      hits += static_cast<uint32_t>(__popcll(gt));
      const unsigned emit = __ballot_sync(0xffffffffu, gt != 0ull);
      if (gt != 0ull) list[nlist + __popc(emit & ((1u << lane) - 1u))] = make_ulonglong2(static_cast<uint64_t>(row), gt);
      nlist += static_cast<uint32_t>(__popc(emit));
    } else {
      pos = write_rows(a, fp, lane, row, gt, c, pos);
      if (valid)
        for (int bit = 0; bit < a.n_in; ++bit) a.votes_out[row * a.n_in + bit] = votes_of(c, bit);
    }
  }
  if (PASS == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hits += __shfl_xor_sync(0xffffffffu, hits, o);
    if (lane == 0) {
      fp.warp_count[gw] = hits;
      fp.warp_rows[gw] = nlist;
    }
  }
}

// Second stage of the small-row path: block b writes the located indices of warps
// [8b, 8b + 8) of the count pass, in ascending order.  Its output offset is the sum of the
// counts of all earlier warps (each block sums them itself: no separate scan).  Every load
// is issued up front.  Votes of the located indices, when asked for, are recounted from
// the global tables.
template <int DV, int NP>
__global__ void __launch_bounds__(kRowWarps * 32) emit_rows_kernel(const RowArgs a, RowTables gt_tables) {
  chain_wait();
  chain_release();
  const FramePtrs fp = frame_ptrs(a);
  gt_tables.bits = fp.det_bits;
  __shared__ unsigned long long red[kRowWarps];
  __shared__ unsigned int wcnt[kRowWarps];
  __shared__ unsigned long long warp_pos[kRowWarps];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t first = static_cast<int64_t>(blockIdx.x) * kRowWarps;
  const int64_t gw = first + wid;
  const bool live = gw < a.warps;
  const ulonglong2* list = fp.row_list + (live ? gw : 0) * a.rows_per_warp;
  // speculative: the first 32 entries of the warp's list (the list has rows_per_warp >= 32 slots)
  const ulonglong2 e0 = live ? list[lane] : make_ulonglong2(0ull, 0ull);
  const unsigned int n = live ? fp.warp_rows[gw] : 0u;
  if (lane == 0) wcnt[wid] = live ? fp.warp_count[gw] : 0u;
  unsigned long long s = 0ull;
  if ((reinterpret_cast<uintptr_t>(fp.warp_count) & 15u) == 0) {
    // four counts a load (first is a multiple of kRowWarps = 8, the counts 16-byte aligned)
    const uint4* wc4 = reinterpret_cast<const uint4*>(fp.warp_count);
#pragma unroll 4
    for (int64_t w = threadIdx.x; w < (first >> 2); w += kRowWarps * 32) {
      const uint4 v = wc4[w];
      s += static_cast<unsigned long long>(v.x) + v.y + v.z + v.w;
    }
  } else {
#pragma unroll 8
    for (int64_t w = threadIdx.x; w < first; w += kRowWarps * 32) s += fp.warp_count[w];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (wid == 0) {
    unsigned long long base = lane < kRowWarps ? red[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) base += __shfl_xor_sync(0xffffffffu, base, o);
    const unsigned long long v = lane < kRowWarps ? wcnt[lane] : 0ull;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane < kRowWarps) warp_pos[lane] = base + incl - v;
    if (lane == kRowWarps - 1 && first + kRowWarps >= a.warps) *fp.d_count = static_cast<int64_t>(base + incl);
  }
  __syncthreads();
  if (!live) return;
  uint64_t pos = warp_pos[wid];
  for (int base = 0; base < static_cast<int>(n); base += 32) {
    const bool act = base + lane < static_cast<int>(n);
    const ulonglong2 e = base == 0 ? (act ? e0 : make_ulonglong2(0ull, 0ull))
                                   : (act ? list[base + lane] : make_ulonglong2(0ull, 0ull));
    uint64_t c[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) c[p] = 0ull;
    if (act && a.located_votes) count_row<DV, NP>(a, gt_tables, static_cast<int64_t>(e.x), c);
    pos = write_rows(a, fp, lane, static_cast<int64_t>(e.x), e.y, c, pos);
  }
}

}  // namespace

cudaError_t launch_count_scan(const uint32_t* counts, int64_t n, uint64_t* offsets, int64_t* total,
                              cudaStream_t stream) {
  stage2_scan_kernel<<<1, 1024, 0, stream>>>(counts, n, offsets, total);
  return cudaGetLastError();
}

cudaError_t launch_vote_scatter(const Geometry& g, const DeviceTables& t, const uint32_t* det_bits,
                                int64_t words_b, uint32_t* votes, cudaStream_t stream) {
  VoteArgs args;
  args.g = g;
  args.t = t;
  args.det_bits = det_bits;
  args.words_b = words_b;
  args.votes = votes;
  const int64_t words = static_cast<int64_t>(g.loops) * words_b;
  int64_t blocks = (words + 7) / 8;  // 8 warps per block
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  vote_scatter_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(args);
  return cudaGetLastError();
}

int64_t stage2_segments(int64_t total_n) { return (total_n + kSegBytes - 1) / kSegBytes; }

cudaError_t launch_stage2(const Geometry& g, int mu, Workspace& ws, uint64_t* located,
                          uint8_t* located_votes, uint8_t* votes_out, int64_t capacity,
                          int64_t* d_count, cudaStream_t stream) {
  const uint32_t mu4 = static_cast<uint32_t>(mu) * 0x01010101u;
  const int64_t segs = ws.segments;
  const unsigned grid = static_cast<unsigned>(segs < 152 * 32 ? segs : 152 * 32);
  stage2_count_kernel<<<grid, kSegThreads, 0, stream>>>(reinterpret_cast<const uint4*>(ws.votes), segs, mu4,
                                                        ws.seg_count);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stage2_scan_kernel<<<1, 1024, 0, stream>>>(ws.seg_count, segs, ws.seg_offset, d_count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stage2_write_kernel<<<grid, kSegThreads, 0, stream>>>(reinterpret_cast<uint4*>(ws.votes), segs,
                                                        static_cast<uint32_t>(mu), mu4, ws.seg_offset, located,
                                                        located_votes, votes_out, g.total_n, capacity);
  return cudaGetLastError();
}

template <int DV, int NP>
cudaError_t small_rows_attr(size_t smem) {
  cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(vote_rows_small_kernel<0, DV, NP>), static_cast<int>(smem));
  if (e == cudaSuccess)
    e = ensure_smem_limit(reinterpret_cast<const void*>(vote_rows_small_kernel<1, DV, NP>), static_cast<int>(smem));
  return e;
}

// Shared memory of the small-row kernels, with their dynamic shared-memory limit raised to match.
static cudaError_t small_rows_smem(const Geometry& g, const VoteRowSchedule& vs, int64_t words_b, size_t* smem) {
  *smem = small_row_layout(g, vs.d_v, vs.b_in, words_b).total;
  cudaError_t e = small_rows_attr<0, 8>(*smem);
  if (e == cudaSuccess) e = small_rows_attr<0, 4>(*smem);
  if (e == cudaSuccess) e = small_rows_attr<1, 8>(*smem);
  if (e == cudaSuccess) e = small_rows_attr<1, 4>(*smem);
  if (e == cudaSuccess) e = small_rows_attr<2, 8>(*smem);
  if (e == cudaSuccess) e = small_rows_attr<2, 4>(*smem);
  if (e == cudaSuccess) e = small_rows_attr<3, 8>(*smem);
  if (e == cudaSuccess) e = small_rows_attr<3, 4>(*smem);
  return e;
}

template <int DV, int NP>
cudaError_t small_rows_run(const RowArgs& a, const RowTables& gtab, size_t smem, bool full, cudaStream_t stream,
                           int nframes) {
  const dim3 blocks(static_cast<unsigned>((a.warps + kSmallWarps - 1) / kSmallWarps), static_cast<unsigned>(nframes));
  cudaError_t e = launch_chained(vote_rows_small_kernel<0, DV, NP>, blocks, dim3(kSmallWarps * 32), smem, stream, a);
  if (e != cudaSuccess) return e;
  if (full) {
    // the full vote array: scan the warp counts, recount and write every row
    stage2_scan_kernel<<<1, 1024, 0, stream>>>(a.warp_count, a.warps, const_cast<uint64_t*>(a.warp_offset), a.d_count);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_chained(vote_rows_small_kernel<1, DV, NP>, blocks, dim3(kSmallWarps * 32), smem, stream, a);
  }
  const dim3 eblocks(static_cast<unsigned>((a.warps + kRowWarps - 1) / kRowWarps), static_cast<unsigned>(nframes));
  return launch_chained(emit_rows_kernel<DV, NP>, eblocks, dim3(kRowWarps * 32), 0, stream, a, gtab);
}

size_t vote_rows_small_smem(const Geometry& g, const VoteRowSchedule& vs, int64_t words_b) {
  return small_row_layout(g, vs.d_v, vs.b_in, words_b).total;
}

cudaError_t vote_rows_small_residency(const Geometry& g, const VoteRowSchedule& vs, int64_t words_b,
                                      int* warps_per_sm) {
  size_t smem = 0;
  cudaError_t e = small_rows_smem(g, vs, words_b, &smem);
  if (e != cudaSuccess) return e;
  int blocks = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, vote_rows_small_kernel<0, 2, 4>, kSmallWarps * 32, smem);
  *warps_per_sm = blocks * kSmallWarps;
  return e;
}

cudaError_t launch_vote_rows(const Geometry& g, const VoteRowSchedule& vs, const DeviceTables& t,
                             const uint32_t* det_bits, int64_t words_b, int mu, uint32_t* warp_count,
                             uint64_t* warp_offset, uint64_t* located, uint8_t* located_votes,
                             uint8_t* votes_out, int64_t capacity, int64_t* d_count, int* err,
                             ulonglong2* row_list, uint32_t* warp_rows, cudaStream_t stream, int nframes,
                             int64_t frame_bits) {
  if (nframes > 1 && (!vs.small || votes_out)) return cudaErrorInvalidValue;  // frames: small rows, no vote array
  if (vs.small) {
    RowArgs a;
    a.frame_bits = frame_bits;
    a.g = g;
    a.t = t;
    a.det_bits = det_bits;
    a.words_b = words_b;
    a.d_v = vs.d_v;
    a.n_in = vs.n_in;
    a.b_in = vs.b_in;
    a.m_in = vs.m_in;
    a.rows = vs.rows;
    a.rows_per_warp = vs.rows_per_warp;
    a.warps = vs.warps;
    a.mu = mu;
    a.warp_count = warp_count;
    a.warp_offset = warp_offset;
    a.located = located;
    a.located_votes = located_votes;
    a.votes_out = votes_out;
    a.capacity = capacity;
    a.err = err;
    a.row_list = row_list;
    a.warp_rows = warp_rows;
    a.d_count = d_count;
    size_t smem = 0;
    cudaError_t e = small_rows_smem(g, vs, words_b, &smem);
    if (e != cudaSuccess) return e;
    RowTables gtab;
    gtab.kb = t.kb16;
    gtab.cand = t.rowmask;
    gtab.bits = det_bits;
    const bool few = g.loops <= 15;  // four counter planes hold the votes
    switch (vs.d_v * 2 + (few ? 1 : 0)) {
      case 0: return small_rows_run<0, 8>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      case 1: return small_rows_run<0, 4>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      case 2: return small_rows_run<1, 8>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      case 3: return small_rows_run<1, 4>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      case 4: return small_rows_run<2, 8>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      case 5: return small_rows_run<2, 4>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      case 6: return small_rows_run<3, 8>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      case 7: return small_rows_run<3, 4>(a, gtab, smem, votes_out != nullptr, stream, nframes);
      default: return cudaErrorInvalidValue;
    }
  }
  RowArgs a;
  a.g = g;
  a.t = t;
  a.err = err;
  a.det_bits = det_bits;
  a.words_b = words_b;
  a.d_v = vs.d_v;
  a.n_in = vs.n_in;
  a.b_in = vs.b_in;
  a.m_in = vs.m_in;
  a.rows = vs.rows;
  a.rows_per_warp = vs.rows_per_warp;
  a.warps = vs.warps;
  a.mu = mu;
  a.warp_count = warp_count;
  a.warp_offset = warp_offset;
  a.located = located;
  a.located_votes = located_votes;
  a.votes_out = votes_out;
  a.capacity = capacity;
  const unsigned blocks = static_cast<unsigned>((vs.warps + kRowWarps - 1) / kRowWarps);
  const size_t cnt_bytes = static_cast<size_t>(kRowWarps) * ((vs.n_in + 3) / 4) * 4;
  const size_t bit_bytes = static_cast<size_t>(g.loops) * words_b * 4;
  const int staged = cnt_bytes + bit_bytes <= 112 * 1024 ? 1 : 0;
  const size_t smem = cnt_bytes + (staged ? bit_bytes : 0);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(vote_rows_kernel<0>), static_cast<int>(smem));
    if (e == cudaSuccess)
      e = ensure_smem_limit(reinterpret_cast<const void*>(vote_rows_kernel<1>), static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  vote_rows_kernel<0><<<blocks, kRowWarps * 32, smem, stream>>>(a, staged);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  stage2_scan_kernel<<<1, 1024, 0, stream>>>(warp_count, vs.warps, warp_offset, d_count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  vote_rows_kernel<1><<<blocks, kRowWarps * 32, smem, stream>>>(a, staged);
  return cudaGetLastError();
}

cudaError_t launch_median(const Geometry& g, const DeviceTables& t, const float2* spectrum,
                          const uint64_t* located, const int64_t* d_count, int64_t capacity,
                          float2* amp, cudaStream_t stream, int nframes) {
  MedianArgs args;
  args.g = g;
  args.t = t;
  args.spectrum = spectrum;
  args.located = located;
  args.d_count = d_count;
  args.capacity = capacity;
  args.amp = amp;
  int64_t blocks = (capacity + kMedianWarps - 1) / kMedianWarps;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  const int L = g.loops;
  const int per_warp = L <= 4 ? 8 : L <= 8 ? 4 : L <= 16 ? 2 : L <= 32 ? 1 : 0;
  if (per_warp > 0) {
    int64_t gb = (capacity + kMedianWarps * per_warp - 1) / (kMedianWarps * per_warp);
    if (gb > 152 * 8) gb = 152 * 8;
    if (gb < 1) gb = 1;
    const dim3 gu(static_cast<unsigned>(gb), static_cast<unsigned>(nframes));
    const dim3 blk(kMedianWarps * 32);
    if (per_warp == 8) return launch_chained(median_group_kernel<4>, gu, blk, 0, stream, args);
    if (per_warp == 4) return launch_chained(median_group_kernel<8>, gu, blk, 0, stream, args);
    if (per_warp == 2) return launch_chained(median_group_kernel<16>, gu, blk, 0, stream, args);
    return launch_chained(median_group_kernel<32>, gu, blk, 0, stream, args);
  }
  return launch_chained(median_kernel, dim3(static_cast<unsigned>(blocks), static_cast<unsigned>(nframes)),
                        dim3(kMedianWarps * 32), 0, stream, args);
}

}  // namespace rsft

// ---------------------------------------------------------------------------
// Second-stage compaction that allocates nothing.
//
// Some callers cannot allocate device memory when they run the second stage:
// a real-time radar loop whose memory is fixed at start-up, code that must not
// call cudaMalloc/cudaFree while other work on the device is in flight (both
// calls can synchronise the device), or a host framework that owns every
// allocation itself.  rsft_stage2_static serves them: it runs the same three
// kernels as the second stage of rsft_execute (count, scan, ordered write) on
// a vote array the caller owns, and keeps its only scratch -- the per-segment
// hit counts and their offsets -- in the fixed array below, which every GPU
// that loads this library holds until the process exits.
namespace rsft {
namespace {

constexpr int64_t kStaticSegments = 16384;  // 16384 segments of 16 KiB: at most 2^28 votes per call
constexpr size_t kStaticOffsetBytes = static_cast<size_t>(kStaticSegments + 1) * sizeof(uint64_t);
constexpr size_t kStaticScratchBytes = kStaticOffsetBytes + static_cast<size_t>(kStaticSegments) * sizeof(uint32_t);

static __device__ __align__(256) unsigned char g_stage2_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;
void* g_static_addr[256] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t static_scratch(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
  if (!g_static_addr[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_stage2_scratch);
    if (e != cudaSuccess) return e;
    g_static_addr[device] = ptr;
  }
  *out = g_static_addr[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace rsft

extern "C" rsft_status rsft_stage2_static(uint8_t* d_votes, int64_t n, int32_t mu, uint64_t* d_located,
                                          uint8_t* d_located_votes, int64_t capacity, int64_t* d_count,
                                          void* stream) {
  using namespace rsft;
  if (!d_votes || !d_count || n <= 0 || capacity < 0 || (capacity > 0 && !d_located)) {
    set_last_error("rsft_stage2_static: NULL pointer or non-positive size");
    return RSFT_ERR_INVALID_ARG;
  }
  if (reinterpret_cast<uintptr_t>(d_votes) % 16 != 0) {
    set_last_error("rsft_stage2_static: d_votes must be 16-byte aligned");
    return RSFT_ERR_INVALID_ARG;
  }
  if (n % (16 * 1024) != 0) {
    set_last_error("rsft_stage2_static: n must be a multiple of 16384 votes");
    return RSFT_ERR_INVALID_ARG;
  }
  if (n / (16 * 1024) > kStaticSegments) {
    set_last_error("rsft_stage2_static: n exceeds the static scratch limit of 268435456 votes");
    return RSFT_ERR_INVALID_ARG;
  }
  if (mu < 0 || mu > 254) {
    set_last_error("rsft_stage2_static: mu must be in [0, 254]");
    return RSFT_ERR_INVALID_ARG;
  }
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  void* scratch = nullptr;
  if (e == cudaSuccess) e = static_scratch(device, &scratch);
  if (e != cudaSuccess) {
    set_last_error((std::string("rsft_stage2_static: scratch lookup: ") + cudaGetErrorString(e)).c_str());
    return RSFT_ERR_CUDA;
  }
  Geometry g{};
  g.total_n = n;
  Workspace ws{};
  ws.votes = reinterpret_cast<uint32_t*>(d_votes);
  ws.segments = n / (16 * 1024);
  ws.seg_offset = static_cast<uint64_t*>(scratch);
  ws.seg_count = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(scratch) + kStaticOffsetBytes);
  e = launch_stage2(g, mu, ws, d_located, d_located_votes, nullptr, capacity, d_count,
                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_last_error((std::string("rsft_stage2_static: ") + cudaGetErrorString(e)).c_str());
    return RSFT_ERR_CUDA;
  }
  return RSFT_OK;
}
