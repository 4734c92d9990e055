// bucket_fft + np_detect: the N-D FFT of every loop's bucket array (eq. (f),
// forward, unnormalised) in shared-memory passes, with first-stage
// Neyman-Pearson detection fused into the last pass: bucket k of loop l is
// detected iff |f-hat_l[k]|^2 > gamma_l (§IV-B, eq. (tpd)); the result is a
// bitmap c_l in {0,1}^B (§IV-C) plus a per-loop count.
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

struct FftArgs {
  Geometry g;
  FftPass ps;
  DeviceTables t;
  const float2* in;
  float2* out;
  uint32_t* det_bits;
  uint32_t* det_count;
  int64_t words_b;
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
      hit = v.x * v.x + v.y * v.y > gamma;
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

}  // namespace

cudaError_t launch_fft_pass(const Geometry& g, const FftPass& ps, const DeviceTables& t,
                            const float2* in, float2* out, uint32_t* det_bits, uint32_t* det_count,
                            int64_t words_b, cudaStream_t stream) {
  FftArgs args;
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
