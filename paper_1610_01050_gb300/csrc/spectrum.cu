// bucket_fft + np_detect: the N-D FFT of every loop's bucket array (eq. (f),
// forward, unnormalised) in shared-memory passes, with first-stage
// Neyman-Pearson detection fused into the last pass: bucket k of loop l is
// detected iff |f-hat_l[k]|^2 > gamma_l (§IV-B, eq. (tpd)); the result is a
// bitmap c_l in {0,1}^B (§IV-C) plus a per-loop count.
//
// With the noise level unknown (estimate mode) the last pass only writes the
// spectrum, and noise_floor_kernel takes each loop's threshold from its own
// bucket powers: under H0 a bucket's power is exponential (eq. (exp)), whose
// median is its mean times ln 2, so gamma_l = lowermedian(P_l) / ln 2 times
// -ln Pfa1-bar.  The lower median (rank floor((B - 1) / 2) ascending) is found
// exactly by a radix select on the powers' bit patterns (non-negative floats
// order as their unsigned bits), then the loop's buckets are tested against it.
//
// Cluster form (one launch, used when the bucket grid allows): the C CTAs of a thread-block
// cluster share one loop's B buckets.  CTA c loads rows [c B_0 / C, (c + 1) B_0 / C) of the
// first dimension and transforms dimensions 1..D-1 of its rows in its own shared memory; after
// a cluster barrier it gathers, through distributed shared memory, the columns
// [c S / C, (c + 1) S / C) of all B_0 rows (S = B / B_0) and transforms dimension 0, then writes
// the spectrum and the detection bits of its columns.  Every transform is radix-2
// decimation in time: the bit reversal is applied where the data is stored into shared memory,
// so each stage is one pass of butterflies between barriers.  With C = 1 one CTA does every
// dimension of its loop in place.
//
// A pass transforms dimensions [da, db) of a slab held in shared memory: the
// slab is `opc` consecutive outer indices x all group indices x `width`
// consecutive inner indices.  Each dimension is an in-place radix-2 DIT
// transform (bit reversal, then log2 B_d butterfly stages) with FP64-derived
// twiddles.  The last pass always holds the last dimension, so its slabs are
// contiguous bucket ranges and detection bits are formed by warp ballots.
#include <cooperative_groups.h>

#include "device.cuh"

namespace cg = cooperative_groups;

namespace rsft {
namespace {

constexpr int kFftThreads = 256;
constexpr int kFloorThreads = 1024;

// Bucket power |v|^2 in one fixed FP32 form, shared by the detection of the last FFT pass and the
// noise-floor kernel, so the threshold is ranked among exactly the values it is compared with.
__device__ __forceinline__ float bucket_power(float2 v) { return __fmaf_rn(v.x, v.x, __fmul_rn(v.y, v.y)); }

struct FftArgs {
  Geometry g;
  FftPass ps;
  DeviceTables t;
  const float2* in;
  float2* out;
  uint32_t* det_bits;
  uint32_t* det_count;
  int64_t words_b;
  int detect;             // last pass: test the buckets against gamma_l (known noise)
};

__device__ __forceinline__ int ilog2(int64_t v) { return 63 - __clzll(v); }

__global__ void __launch_bounds__(kFftThreads) fft_pass_kernel(const FftArgs a) {
  extern __shared__ float2 s[];
  const Geometry& g = a.g;
  const FftPass& ps = a.ps;
  const int l = static_cast<int>(blockIdx.x / ps.ctas_per_loop);
  const int64_t q = blockIdx.x % ps.ctas_per_loop;
  const int64_t inner_slabs = ps.inner / ps.width;
  const int64_t o0 = (q / inner_slabs) * ps.outer_per_cta;
  const int64_t i0 = (q % inner_slabs) * ps.width;
  const int64_t S = ps.outer_per_cta * ps.group * ps.width;
  const int lw = ilog2(ps.width), lgp = ilog2(ps.group);
  const float2* src = a.in + static_cast<int64_t>(l) * g.total_b;

  // load: slab element e = ((oo * group) + gi) * width + w
  for (int64_t e = threadIdx.x; e < S; e += kFftThreads) {
    const int64_t w = e & (ps.width - 1);
    const int64_t gi = (e >> lw) & (ps.group - 1);
    const int64_t oo = e >> (lw + lgp);
    s[e] = src[((o0 + oo) * ps.group + gi) * ps.inner + i0 + w];
  }
  __syncthreads();

  // transform dimensions [da, db); stride of dimension d in the slab
  for (int d = ps.da; d < ps.db; ++d) {
    const int64_t n = g.b[d];
    if (n == 1) continue;
    const int ln = g.log_b[d];
    int64_t st = ps.width;
    for (int e2 = d + 1; e2 < ps.db; ++e2) st *= g.b[e2];
    const int lst = ilog2(st);
    // bit reversal along d
    for (int64_t e = threadIdx.x; e < S; e += kFftThreads) {
      const int64_t k = (e >> lst) & (n - 1);
      const int64_t rk = __brevll(static_cast<unsigned long long>(k)) >> (64 - ln);
      if (k < rk) {
        const int64_t e2 = e + ((rk - k) << lst);
        const float2 tmp = s[e];
        s[e] = s[e2];
        s[e2] = tmp;
      }
    }
    __syncthreads();
    const float2* tw = a.t.twiddle[d];
    for (int lh = 0; lh < ln; ++lh) {
      const int64_t h = int64_t(1) << lh;
      for (int64_t bf = threadIdx.x; bf < (S >> 1); bf += kFftThreads) {
        const int64_t lo = bf & (st - 1);
        const int64_t t = bf >> lst;              // [lines * n / 2]
        const int64_t b = t & ((n >> 1) - 1);     // butterfly within the line
        const int64_t line = t >> (ln - 1);
        const int64_t pos = b & (h - 1);
        const int64_t grp = b >> lh;
        const int64_t i0s = ((line << ln) + (grp << (lh + 1)) + pos) * st + lo;
        const int64_t i1s = i0s + (h << lst);
        const float2 w = __ldg(tw + (pos << (ln - 1 - lh)));
        const float2 x0 = s[i0s], x1 = s[i1s];
        const float2 y = make_float2(x1.x * w.x - x1.y * w.y, x1.x * w.y + x1.y * w.x);
        s[i0s] = make_float2(x0.x + y.x, x0.y + y.y);
        s[i1s] = make_float2(x0.x - y.x, x0.y - y.y);
      }
      __syncthreads();
    }
  }

  float2* dst = a.out + static_cast<int64_t>(l) * g.total_b;
  if (!ps.last) {
    for (int64_t e = threadIdx.x; e < S; e += kFftThreads) {
      const int64_t w = e & (ps.width - 1);
      const int64_t gi = (e >> lw) & (ps.group - 1);
      const int64_t oo = e >> (lw + lgp);
      dst[((o0 + oo) * ps.group + gi) * ps.inner + i0 + w] = s[e];
    }
    return;
  }
  // last pass: inner == width == 1, the slab is the contiguous bucket range [base, base + S)
  if (!a.detect) {
    for (int64_t e = threadIdx.x; e < S; e += kFftThreads) dst[o0 * ps.group + e] = s[e];
    return;
  }
  const float gamma = a.t.gamma[l];
  const int64_t base = o0 * ps.group;
  uint32_t* bits = a.det_bits + static_cast<int64_t>(l) * a.words_b;
  const int lane = threadIdx.x & 31;
  for (int64_t e0 = 0; e0 < S; e0 += kFftThreads) {
    const int64_t e = e0 + threadIdx.x;
    bool hit = false;
    if (e < S) {
      const float2 v = s[e];
      dst[base + e] = v;
      hit = bucket_power(v) > gamma;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    if (lane == 0 && ballot) {
      const int64_t k0 = base + e - lane;  // bucket of lane 0 (a multiple of 32 when S >= 32)
      if ((k0 & 31) == 0) {
        atomicOr(bits + (k0 >> 5), ballot);
      } else {
        for (int i = 0; i < 32; ++i)
          if ((ballot >> i) & 1u) atomicOr(bits + ((k0 + i) >> 5), 1u << ((k0 + i) & 31));
      }
      atomicAdd(a.det_count + l, static_cast<uint32_t>(__popc(ballot)));
    }
  }
}

struct ClusterFftArgs {
  Geometry g;
  DeviceTables t;
  const float2* in;      // [L][B] folded buckets
  float2* out;           // [L][B] spectrum
  uint32_t* det_bits;
  uint32_t* det_count;
  int64_t words_b;
  int csize;             // C: CTAs per loop (a cluster)
  int detect;
  int64_t frame_bits;    // frames (blockIdx.y): detection words between consecutive frames
  float* gamma_out;      // non-null: estimate mode, gamma_l from the loop's own bucket powers ([frames][L])
  float floor_factor;    // -ln Pfa1-bar / ln 2 (estimate mode)
};

// Reverse the bits of each dimension's digit of a row-major index over dimensions [d0, D).
__device__ __forceinline__ uint32_t digit_reverse(uint32_t q, const Geometry& g, int d0) {
  uint32_t out = 0u;
  int shift = 0;
#pragma unroll
  for (int d = kMaxDim - 1; d >= 0; --d) {
    if (d < d0 || d >= g.ndim) continue;
    const int lb = g.log_b[d];
    const uint32_t dig = (q >> shift) & ((1u << lb) - 1u);
    out |= (lb ? (__brev(dig) >> (32 - lb)) : 0u) << shift;
    shift += lb;
  }
  return out | ((q >> shift) << shift);  // digits of dimensions below d0 pass through
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// All decimation-in-time stages of dimension d (size n = 2^ln, element stride 2^lst) of an
// E-element shared-memory buffer whose input along d is in bit-reversed order, several radix-2
// stages per pass between barriers: three while three or more remain (except four, taken as
// two and two), then two, then one.  A radix-2^3 butterfly on eight elements spaced h apart:
// stage h pairs (a0, a1), (a2, a3), ... with W_2h^p; stage 2h pairs (b0, b2), (b4, b6) with
// W_4h^p and (b1, b3), (b5, b7) with W_4h^(p + h) = -j W_4h^p; stage 4h pairs (c_k, c_k+4) with
// W_8h^(p + k h) = W_8h^p W_8^k.  A radix-2^2 butterfly is its first two stages on four
// elements.  tw[k] = e^{-j 2 pi k / n}.
__device__ __forceinline__ void dit_dimension(float2* buf, uint32_t E, int ln, int lst, const float2* __restrict__ tw) {
  const uint32_t smask = (1u << lst) - 1u;
  const float r2 = 0.70710678118654752f;  // 1 / sqrt 2
  int lh = 0;
  for (; lh + 2 < ln && ln - lh != 4; lh += 3) {
    const uint32_t eighth = E >> 3;
    for (uint32_t qi = threadIdx.x; qi < eighth; qi += blockDim.x) {
      const uint32_t low = qi & smask;
      const uint32_t t = qi >> lst;
      const uint32_t b = t & ((1u << (ln - 3)) - 1u);
      const uint32_t line = t >> (ln - 3);
      const uint32_t pos = b & ((1u << lh) - 1u);
      const uint32_t grp = b >> lh;
      const uint32_t i0 = (((line << ln) + (grp << (lh + 3)) + pos) << lst) + low;
      const uint32_t hs = 1u << (lh + lst);
      const float2 w1 = tw[pos << (ln - 1 - lh)];  // W_2h^pos
      const float2 w2 = tw[pos << (ln - 2 - lh)];  // W_4h^pos
      const float2 w3 = tw[pos << (ln - 3 - lh)];  // W_8h^pos
      float2 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = buf[i0 + k * hs];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {  // stage h
        const float2 y = cmulf(w1, v[k + 1]);
        v[k + 1] = make_float2(v[k].x - y.x, v[k].y - y.y);
        v[k] = make_float2(v[k].x + y.x, v[k].y + y.y);
      }
#pragma unroll
      for (int k = 0; k < 8; k += 4) {  // stage 2h
        const float2 y0 = cmulf(w2, v[k + 2]);
        const float2 u1 = cmulf(w2, v[k + 3]);
        const float2 y1 = make_float2(u1.y, -u1.x);  // -j W_4h^pos
        v[k + 2] = make_float2(v[k].x - y0.x, v[k].y - y0.y);
        v[k] = make_float2(v[k].x + y0.x, v[k].y + y0.y);
        v[k + 3] = make_float2(v[k + 1].x - y1.x, v[k + 1].y - y1.y);
        v[k + 1] = make_float2(v[k + 1].x + y1.x, v[k + 1].y + y1.y);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // stage 4h: W_8h^pos W_8^k
        const float2 u = cmulf(w3, v[k + 4]);
        float2 y;
        if (k == 0) y = u;
        else if (k == 1) y = make_float2((u.x + u.y) * r2, (u.y - u.x) * r2);
        else if (k == 2) y = make_float2(u.y, -u.x);
        else y = make_float2((u.y - u.x) * r2, -(u.x + u.y) * r2);
        buf[i0 + k * hs] = make_float2(v[k].x + y.x, v[k].y + y.y);
        buf[i0 + (k + 4) * hs] = make_float2(v[k].x - y.x, v[k].y - y.y);
      }
    }
    __syncthreads();
  }
  for (; lh + 1 < ln; lh += 2) {
    const uint32_t quarter = E >> 2;
    for (uint32_t qi = threadIdx.x; qi < quarter; qi += blockDim.x) {
      const uint32_t low = qi & smask;
      const uint32_t t = qi >> lst;                        // [lines * n / 4]
      const uint32_t b = t & ((1u << (ln - 2)) - 1u);
      const uint32_t line = t >> (ln - 2);
      const uint32_t pos = b & ((1u << lh) - 1u);          // position within a block of 4h
      const uint32_t grp = b >> lh;
      const uint32_t i0 = (((line << ln) + (grp << (lh + 2)) + pos) << lst) + low;
      const uint32_t hs = 1u << (lh + lst);
      const float2 w1 = tw[pos << (ln - 1 - lh)];          // W_2h^pos
      const float2 w2 = tw[pos << (ln - 2 - lh)];          // W_4h^pos
      const float2 a0 = buf[i0], a1 = buf[i0 + hs], a2 = buf[i0 + 2 * hs], a3 = buf[i0 + 3 * hs];
      const float2 y1 = cmulf(w1, a1), y3 = cmulf(w1, a3);
      const float2 b0 = make_float2(a0.x + y1.x, a0.y + y1.y), b1 = make_float2(a0.x - y1.x, a0.y - y1.y);
      const float2 b2 = make_float2(a2.x + y3.x, a2.y + y3.y), b3 = make_float2(a2.x - y3.x, a2.y - y3.y);
      const float2 z2 = cmulf(w2, b2);
      const float2 u3 = cmulf(w2, b3);
      const float2 z3 = make_float2(u3.y, -u3.x);          // -j W_4h^pos b3
      buf[i0] = make_float2(b0.x + z2.x, b0.y + z2.y);
      buf[i0 + 2 * hs] = make_float2(b0.x - z2.x, b0.y - z2.y);
      buf[i0 + hs] = make_float2(b1.x + z3.x, b1.y + z3.y);
      buf[i0 + 3 * hs] = make_float2(b1.x - z3.x, b1.y - z3.y);
    }
    __syncthreads();
  }
  if (lh < ln) {  // the last stage, when log2 n is odd
    const uint32_t half = E >> 1;
    for (uint32_t bf = threadIdx.x; bf < half; bf += blockDim.x) {
      const uint32_t low = bf & smask;
      const uint32_t t = bf >> lst;
      const uint32_t b = t & ((1u << (ln - 1)) - 1u);
      const uint32_t line = t >> (ln - 1);
      const uint32_t pos = b & ((1u << lh) - 1u);
      const uint32_t grp = b >> lh;
      const uint32_t i0 = (((line << ln) + (grp << (lh + 1)) + pos) << lst) + low;
      const uint32_t i1 = i0 + (1u << (lh + lst));
      const float2 w = tw[pos << (ln - 1 - lh)];
      const float2 x0 = buf[i0], x1 = buf[i1];
      const float2 y = cmulf(w, x1);
      buf[i0] = make_float2(x0.x + y.x, x0.y + y.y);
      buf[i1] = make_float2(x0.x - y.x, x0.y - y.y);
    }
    __syncthreads();
  }
}

// Spectrum and detections of the E buffer elements of a CTA: element e is row e >> lq (of 2^lq
// elements each) and column e & (2^lq - 1) of the CTA's column block, i.e. bucket
// ((e >> lq) << lS) + col0 + (e & (2^lq - 1)) of loop l.  Rows of at least 32 elements keep a
// warp's 32 consecutive elements on one aligned detection word.
__device__ __forceinline__ void store_block(const ClusterFftArgs& a, int l, const float2* src, uint32_t E, int lq,
                                            int lS, uint32_t col0, float gamma, uint32_t* hits, bool store = true,
                                            bool detect_now = false) {
  const bool detect = detect_now || a.detect;
  const int64_t f = blockIdx.y;
  float2* dst = a.out + (f * a.g.loops + l) * a.g.total_b;
  uint32_t* bits = a.det_bits + f * a.frame_bits + static_cast<int64_t>(l) * a.words_b;
  const int lane = threadIdx.x & 31;
  const uint32_t qmask = (1u << lq) - 1u;
  for (uint32_t e0 = 0; e0 < E; e0 += blockDim.x) {
    const uint32_t e = e0 + threadIdx.x;
    const uint32_t k = ((e >> lq) << lS) + col0 + (e & qmask);
    bool hit = false;
    if (e < E) {
      const float2 v = src[e];
      if (store) dst[k] = v;
      hit = detect && bucket_power(v) > gamma;
    }
    if (!detect) continue;
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    if (lane == 0 && ballot) {
      const uint32_t kw = k;                 // bucket of lane 0
      if ((kw & 31u) == 0u && (qmask >= 31u || E <= 32u)) {
        atomicOr(bits + (kw >> 5), ballot);
      } else {
        for (int i = 0; i < 32; ++i)
          if ((ballot >> i) & 1u) {
            const uint32_t ki = (((e + i) >> lq) << lS) + col0 + ((e + i) & qmask);   // lane 0: e is lane 0's
            atomicOr(bits + (ki >> 5), 1u << (ki & 31u));
          }
      }
      atomicAdd(hits, static_cast<uint32_t>(__popc(ballot)));
    }
  }
}

// Lower median (rank floor((B - 1) / 2)) of the power bit patterns of a loop's B buckets, held
// E apiece in the shared memory of the C CTAs of a cluster: four passes over 8-bit digits, most
// significant first (non-negative floats order as their bit patterns); each CTA histograms its
// own elements whose high digits match the prefix, then every CTA sums the C histograms through
// distributed shared memory (hist holds 512 words: the CTA's own bins, then the cluster's
// totals) and takes the same digit.  Returns the selected pattern.
__device__ __forceinline__ uint32_t cluster_lower_median(const float2* buf, uint32_t E, uint32_t B, int C,
                                                         uint32_t* hist, uint32_t* pick) {
  cg::cluster_group cluster = cg::this_cluster();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t prefix = 0u, rank = (B - 1u) / 2u;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    const uint32_t hi_mask = pass == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (uint32_t e0 = 0; e0 < E; e0 += blockDim.x) {
      const uint32_t e = e0 + threadIdx.x;
      bool take = false;
      uint32_t digit = 0u;
      if (e < E) {
        const uint32_t key = __float_as_uint(bucket_power(buf[e]));
        take = (key & hi_mask) == prefix;
        digit = (key >> shift) & 255u;
      }
      const unsigned active = __ballot_sync(0xffffffffu, take);
      if (take) {
        const unsigned peers = __match_any_sync(active, digit);
        if (lane == __ffs(peers) - 1) atomicAdd(&hist[digit], static_cast<uint32_t>(__popc(peers)));
      }
    }
    if (C > 1) {
      cluster.sync();  // every CTA's histogram is complete
      // thread b sums bin b over the cluster (C independent remote loads), into this CTA's totals
      for (uint32_t b = threadIdx.x; b < 256; b += blockDim.x) {
        uint32_t t = 0u;
        for (int r = 0; r < C; ++r) t += cluster.map_shared_rank(hist, r)[b];
        hist[256 + b] = t;
      }
      cluster.sync();  // the histograms are read before anyone moves on (the next pass clears them)
    } else {
      __syncthreads();
    }
    const uint32_t* tot = C > 1 ? hist + 256 : hist;
    if (warp == 0) {
      // lane q holds bins [8q, 8q + 8): find the bin where the running count passes rank
      uint32_t c[8], sum = 0u;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        c[j] = tot[lane * 8 + j];
        sum += c[j];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint32_t excl = incl - sum;
      if (excl <= rank && rank < incl) {
        uint32_t run = excl;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (run <= rank && rank < run + c[j]) {
            pick[0] = static_cast<uint32_t>(lane * 8 + j);
            pick[1] = run;
          }
          run += c[j];
        }
      }
    }
    __syncthreads();  // pick[] is written
    prefix |= pick[0] << shift;
    rank -= pick[1];
    __syncthreads();  // pick[] is rewritten by the next pass
  }
  return prefix;
}

__global__ void __launch_bounds__(512) fft_cluster_kernel(const ClusterFftArgs a) {
  extern __shared__ __align__(16) float2 sbuf[];
  __shared__ uint32_t hits;
  const Geometry& g = a.g;
  const int C = a.csize;
  const int l = static_cast<int>(blockIdx.x) / C;
  const uint32_t c = blockIdx.x % C;           // rank in the cluster (clusters run along x)
  const uint32_t B = static_cast<uint32_t>(g.total_b);
  const uint32_t E = B / C;                     // this CTA's elements in each phase
  const uint32_t S = B >> g.log_b[0];           // elements of one row of dimension 0
  const int lS = 31 - __clz(S);
  const float2* src = a.in + (static_cast<int64_t>(blockIdx.y) * g.loops + l) * B + static_cast<int64_t>(c) * E;
  const int d_first = C == 1 ? 0 : 1;           // dimensions transformed in place
  if (threadIdx.x == 0) hits = 0u;
  // every dimension's twiddles e^{-j 2 pi k / B_d}, k < B_d / 2, after the two data buffers
  float2* twb = sbuf + (C > 1 ? 2 * E : E);
  const float2* tws[kMaxDim];
  {
    uint32_t off = 0;
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d) {
      tws[d] = twb + off;
      if (d < g.ndim && g.log_b[d] > 0) {
        const uint32_t nh = 1u << (g.log_b[d] - 1);
        for (uint32_t k = threadIdx.x; k < nh; k += blockDim.x) twb[off + k] = __ldg(a.t.twiddle[d] + k);
        off += nh;
      }
    }
  }
  // (the twiddles are the plan's: staged while the previous kernel of the chain finishes)
  chain_wait();
  chain_release();
  // phase 1: rows [c E / S, (c + 1) E / S) of the loop, bit-reversed along dimensions d_first..D-1
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) sbuf[digit_reverse(e, g, d_first)] = src[e];
  __syncthreads();
  for (int d = g.ndim - 1; d >= d_first; --d)
    if (g.log_b[d] > 0)
      dit_dimension(sbuf, E, g.log_b[d], g.b_shift[d], tws[d]);
  const float gamma = a.detect ? a.t.gamma[l] : 0.f;
  __shared__ uint32_t sel_hist[512];
  __shared__ uint32_t sel_pick[2];
  if (C == 1) {
    const int lB = 31 - __clz(B);                // the loop as one row: bucket k = e
    store_block(a, l, sbuf, B, lB, lB, 0u, gamma, &hits);
    if (a.gamma_out) {
      // estimate mode: the noise floor from this loop's own bucket powers, then its detections
      const float gl = __uint_as_float(cluster_lower_median(sbuf, B, B, 1, sel_hist, sel_pick)) * a.floor_factor;
      if (threadIdx.x == 0) a.gamma_out[static_cast<int64_t>(blockIdx.y) * g.loops + l] = gl;
      store_block(a, l, sbuf, B, lB, lB, 0u, gl, &hits, false, true);
    }
  } else {
    // phase 2: columns [c Q, (c + 1) Q) of every row of dimension 0, from the cluster's shared memory
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();                              // every CTA's phase-1 rows are complete and visible
    const uint32_t Q = S / C;
    const uint32_t rows_per = E >> lS;           // rows of dimension 0 held by each CTA
    const int lq = 31 - __clz(Q);
    const int lb0 = g.log_b[0];
    float2* gbuf = sbuf + E;
    for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) {
      const uint32_t row = e >> lq, q = e & (Q - 1u);
      const uint32_t owner = row / rows_per;
      const float2* remote = cluster.map_shared_rank(sbuf, owner);
      const uint32_t rrev = lb0 ? (__brev(row) >> (32 - lb0)) : 0u;
      gbuf[(rrev << lq) + q] = remote[((row - owner * rows_per) << lS) + c * Q + q];
    }
    cluster.sync();                              // no CTA leaves while others still read its rows
    if (lb0 > 0) dit_dimension(gbuf, E, lb0, lq, tws[0]);
    store_block(a, l, gbuf, E, lq, lS, c * Q, gamma, &hits);
    if (a.gamma_out) {
      // estimate mode: the noise floor from the cluster's bucket powers, then this CTA's detections
      const float gl = __uint_as_float(cluster_lower_median(gbuf, E, B, C, sel_hist, sel_pick)) * a.floor_factor;
      if (c == 0 && threadIdx.x == 0) a.gamma_out[static_cast<int64_t>(blockIdx.y) * g.loops + l] = gl;
      store_block(a, l, gbuf, E, lq, lS, c * Q, gl, &hits, false, true);
    }
  }
  if (a.detect || a.gamma_out) {
    __syncthreads();
    if (threadIdx.x == 0 && hits) atomicAdd(a.det_count + static_cast<int64_t>(blockIdx.y) * g.loops + l, hits);
  }
}

struct FloorArgs {
  const float2* spectrum;  // [L][B]
  int64_t total_b;
  int64_t words_b;
  float factor;            // -ln Pfa1-bar / ln 2
  int keys_in_smem;        // the B power patterns fit in shared memory (read the spectrum once)
  float* gamma_out;        // [L] thresholds used
  uint32_t* det_bits;      // [L][words_b], zero on entry
  uint32_t* det_count;     // [L]
  int64_t frame_bits;      // frames (blockIdx.y): detection words between consecutive frames
  int loops;               // L (per frame)
};

// One CTA per loop: radix select of the lower median of the B bucket powers (four 8-bit digits,
// most significant first, over the powers' bit patterns), gamma_l = median * factor, then the
// detection bitmap and count of the loop.
__global__ void __launch_bounds__(kFloorThreads) noise_floor_kernel(const FloorArgs a) {
  extern __shared__ uint32_t keys[];
  __shared__ uint32_t hist[256];
  __shared__ uint32_t pick[2];   // selected digit, count of smaller keys under the prefix
  __shared__ uint32_t hits;
  const int l = blockIdx.x;
  const int64_t fl = static_cast<int64_t>(blockIdx.y) * a.loops + l;   // frame-major loop index
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t B = a.total_b;
  const float2* sp = a.spectrum + fl * B;
  uint32_t prefix = 0u;
  uint32_t rank = static_cast<uint32_t>((B - 1) / 2);
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    const uint32_t hi_mask = pass == 0 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (int i = tid; i < 256; i += kFloorThreads) hist[i] = 0u;
    __syncthreads();
    for (int64_t e0 = 0; e0 < B; e0 += kFloorThreads) {
      const int64_t e = e0 + tid;
      bool take = false;
      uint32_t digit = 0u;
      if (e < B) {
        uint32_t key;
        if (pass > 0 && a.keys_in_smem) {
          key = keys[e];
        } else {
          key = __float_as_uint(bucket_power(sp[e]));
          if (a.keys_in_smem) keys[e] = key;
        }
        take = (key & hi_mask) == prefix;
        digit = (key >> shift) & 255u;
      }
      const unsigned active = __ballot_sync(0xffffffffu, take);
      if (take) {
        const unsigned peers = __match_any_sync(active, digit);
        if (lane == __ffs(peers) - 1) atomicAdd(&hist[digit], static_cast<uint32_t>(__popc(peers)));
      }
    }
    __syncthreads();
    if (warp == 0) {
      // lane q holds bins [8q, 8q + 8): find the bin where the running count passes `rank`
      uint32_t c[8], sum = 0u;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        c[j] = hist[lane * 8 + j];
        sum += c[j];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint32_t excl = incl - sum;
      if (excl <= rank && rank < incl) {
        uint32_t run = excl;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (run <= rank && rank < run + c[j]) {
            pick[0] = static_cast<uint32_t>(lane * 8 + j);
            pick[1] = run;
          }
          run += c[j];
        }
      }
    }
    __syncthreads();
    prefix |= pick[0] << shift;
    rank -= pick[1];
    __syncthreads();  // pick[] is rewritten by the next pass
  }
  const float gamma = __uint_as_float(prefix) * a.factor;
  if (tid == 0) {
    a.gamma_out[fl] = gamma;
    hits = 0u;
  }
  __syncthreads();
  uint32_t* bits = a.det_bits + static_cast<int64_t>(blockIdx.y) * a.frame_bits + static_cast<int64_t>(l) * a.words_b;
  uint32_t mine = 0u;
  for (int64_t e0 = 0; e0 < B; e0 += kFloorThreads) {
    const int64_t e = e0 + tid;
    bool hit = false;
    if (e < B) hit = (a.keys_in_smem ? __uint_as_float(keys[e]) : bucket_power(sp[e])) > gamma;
    const unsigned ballot = __ballot_sync(0xffffffffu, hit);
    if (lane == 0 && e0 + warp * 32 < B) bits[(e0 >> 5) + warp] = ballot;   // e0 + 32 warp is a word start
    mine += hit ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if (lane == 0 && mine) atomicAdd(&hits, mine);
  __syncthreads();
  if (tid == 0) a.det_count[fl] = hits;
}

}  // namespace

cudaError_t launch_noise_floor(const Geometry& g, const float2* spectrum, float factor, float* gamma_out,
                               uint32_t* det_bits, uint32_t* det_count, int64_t words_b, cudaStream_t stream,
                               int nframes, int64_t frame_bits) {
  FloorArgs args;
  args.frame_bits = frame_bits;
  args.loops = g.loops;
  args.spectrum = spectrum;
  args.total_b = g.total_b;
  args.words_b = words_b;
  args.factor = factor;
  args.gamma_out = gamma_out;
  args.det_bits = det_bits;
  args.det_count = det_count;
  args.keys_in_smem = g.total_b <= 32768 ? 1 : 0;
  const int smem = args.keys_in_smem ? static_cast<int>(g.total_b * 4) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(noise_floor_kernel), smem);
    if (e != cudaSuccess) return e;
  }
  noise_floor_kernel<<<dim3(g.loops, nframes), kFloorThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

bool fft_cluster_valid(const Geometry& g, int c) {
  const int64_t B = g.total_b;
  const int64_t S = B / g.b[0];
  if (B < 2 || B > (int64_t(1) << 20) || c < 1 || c > 8 || (c & (c - 1))) return false;
  int64_t twiddles = 0;
  for (int d = 0; d < g.ndim; ++d) twiddles += g.b[d] / 2;
  if (twiddles > 8192 || c > g.b[0] || c > S) return false;
  if (c == 1) return B <= 16384;                // one CTA holds the loop in place (128 KiB)
  return B / c <= 8192 && S / c >= 32;          // two buffers of B / C; whole detection words per run
}

int fft_cluster_size(const Geometry& g) {
  int64_t c = g.total_b / 2048;  // about 2048 buckets per CTA
  if (c < 1) c = 1;
  if (c > 8) c = 8;
  for (; c >= 1; c >>= 1)
    if (fft_cluster_valid(g, static_cast<int>(c))) return static_cast<int>(c);
  return 0;
}

cudaError_t launch_fft_cluster(const Geometry& g, const DeviceTables& t, const float2* in, float2* out,
                               uint32_t* det_bits, uint32_t* det_count, int64_t words_b, bool detect,
                               cudaStream_t stream, int nframes, int64_t frame_bits, int csize_req, int threads_req,
                               float* gamma_out, float floor_factor) {
  const int csize = csize_req > 0 ? csize_req : fft_cluster_size(g);
  if (csize < 1 || !fft_cluster_valid(g, csize)) return cudaErrorInvalidConfiguration;
  if (gamma_out && detect) return cudaErrorInvalidValue;  // one detection per launch: known or estimated
  if (threads_req != 0 && threads_req != 256 && threads_req != 512) return cudaErrorInvalidValue;
  ClusterFftArgs args;
  args.g = g;
  args.t = t;
  args.in = in;
  args.out = out;
  args.det_bits = det_bits;
  args.det_count = det_count;
  args.words_b = words_b;
  args.csize = csize;
  args.detect = detect ? 1 : 0;
  args.frame_bits = frame_bits;
  args.gamma_out = gamma_out;
  args.floor_factor = floor_factor;
  const int64_t E = g.total_b / csize;
  int64_t twiddles = 0;
  for (int d = 0; d < g.ndim; ++d) twiddles += g.b[d] / 2;
  const int smem = static_cast<int>((E * (csize > 1 ? 2 : 1) + twiddles) * sizeof(float2));
  cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(fft_cluster_kernel), smem > 48 * 1024 ? smem : 48 * 1024);
  if (e != cudaSuccess) return e;
  const int threads = threads_req > 0 ? threads_req : (E >= 2048 ? 512 : 256);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(g.loops * csize), static_cast<unsigned>(nframes));
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = static_cast<size_t>(smem);
  cfg.stream = stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(csize);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // chained (chain_wait first)
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = t_chain_launches ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, fft_cluster_kernel, args);
}

cudaError_t launch_fft_pass(const Geometry& g, const FftPass& ps, const DeviceTables& t,
                            const float2* in, float2* out, uint32_t* det_bits, uint32_t* det_count,
                            int64_t words_b, bool detect, cudaStream_t stream) {
  FftArgs args;
  args.detect = detect ? 1 : 0;
  args.g = g;
  args.ps = ps;
  args.t = t;
  args.in = in;
  args.out = out;
  args.det_bits = det_bits;
  args.det_count = det_count;
  args.words_b = words_b;
  const int64_t slab = ps.outer_per_cta * ps.group * ps.width;
  const int smem = static_cast<int>(slab * sizeof(float2));
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_smem_limit(reinterpret_cast<const void*>(fft_pass_kernel), smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t ctas = ps.ctas_per_loop * g.loops;
  fft_pass_kernel<<<static_cast<unsigned>(ctas), kFftThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace rsft
