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
// A pass transforms dimensions [da, db) of a slab held in shared memory: the
// slab is `opc` consecutive outer indices x all group indices x `width`
// consecutive inner indices.  Each dimension is an in-place radix-2 DIT
// transform (bit reversal, then log2 B_d butterfly stages) with FP64-derived
// twiddles.  The last pass always holds the last dimension, so its slabs are
// contiguous bucket ranges and detection bits are formed by warp ballots.
#include "device.cuh"

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

struct FloorArgs {
  const float2* spectrum;  // [L][B]
  int64_t total_b;
  int64_t words_b;
  float factor;            // -ln Pfa1-bar / ln 2
  int keys_in_smem;        // the B power patterns fit in shared memory (read the spectrum once)
  float* gamma_out;        // [L] thresholds used
  uint32_t* det_bits;      // [L][words_b], zero on entry
  uint32_t* det_count;     // [L]
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
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t B = a.total_b;
  const float2* sp = a.spectrum + static_cast<int64_t>(l) * B;
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
    a.gamma_out[l] = gamma;
    hits = 0u;
  }
  __syncthreads();
  uint32_t* bits = a.det_bits + static_cast<int64_t>(l) * a.words_b;
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
  if (tid == 0) a.det_count[l] = hits;
}

}  // namespace

cudaError_t launch_noise_floor(const Geometry& g, const float2* spectrum, float factor, float* gamma_out,
                               uint32_t* det_bits, uint32_t* det_count, int64_t words_b, cudaStream_t stream) {
  FloorArgs args;
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
    cudaError_t e = cudaFuncSetAttribute(noise_floor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  noise_floor_kernel<<<g.loops, kFloorThreads, smem, stream>>>(args);
  return cudaGetLastError();
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
    cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t ctas = ps.ctas_per_loop * g.loops;
  fft_pass_kernel<<<static_cast<unsigned>(ctas), kFftThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace rsft
