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

constexpr int kMedianWarps = 4;

// One warp per located index; per-loop values in shared memory, median by rank.
__global__ void __launch_bounds__(kMedianWarps * 32) median_kernel(const MedianArgs a) {
  __shared__ float vre[kMedianWarps][256];
  __shared__ float vim[kMedianWarps][256];
  __shared__ float sel[kMedianWarps][4];
  const Geometry& g = a.g;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t count = *a.d_count;
  if (count > a.capacity) count = a.capacity;
  const int L = g.loops;
  const int lo_rank = (L - 1) / 2, hi_rank = L / 2;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * kMedianWarps + wid; q < count;
       q += static_cast<int64_t>(gridDim.x) * kMedianWarps) {
    const uint64_t i = a.located[q];
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
      const float2 f = a.spectrum[static_cast<int64_t>(l) * g.total_b + k];
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
    if (lane == 0) a.amp[q] = make_float2(0.5f * (sel[wid][0] + sel[wid][1]), 0.5f * (sel[wid][2] + sel[wid][3]));
    __syncwarp();
  }
}

}  // namespace

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

cudaError_t launch_median(const Geometry& g, const DeviceTables& t, const float2* spectrum,
                          const uint64_t* located, const int64_t* d_count, int64_t capacity,
                          float2* amp, cudaStream_t stream) {
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
  median_kernel<<<static_cast<unsigned>(blocks), kMedianWarps * 32, 0, stream>>>(args);
  return cudaGetLastError();
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
