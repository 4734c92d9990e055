// Bucket-domain refinement of K off-grid tones (beyond the paper, which recovers grid
// locations only, §I).  The loss compares, for every loop l, the cube's folded buckets
// F_l (the fold of Algorithm 1, in bucket order j) with those of the tone model
// s(t) = sum_k a_k exp(j 2 pi f_k . t):
//     E = sum_l sum_j |F_l[j] - fold_l(s)[j]|^2.
// The fold weight a_l(s) = prod_d w-bar_d(sigma_d^{-1} s_d) w_d(s_d) and every tone factor
// over dimensions, so a tone's folded contribution to source residue x (j = sigma^{-1} x)
// is a_k prod_d g_{l,d,k}(x_d) with
//     g_{l,d,k}(x) = sum_m a_{l,d}(x + B_d m) exp(j 2 pi f_kd (x + B_d m)),
// and dE/dtheta = -2 Re sum conj(R) dM/dtheta needs only the per-dimension responses g, their
// frequency derivatives g' (the factor j 2 pi s inside the sum) and one contraction of the
// residual R per (loop, tone): the adjoint of the fold applied to R, contracted with the
// synthesis Jacobian, without forming N-point fields.  Phases f s are reduced exactly in
// 64-bit fixed point before the FP32 sine and cosine.
#include <algorithm>

#include "device.cuh"

namespace rsft {
namespace {

constexpr int kRefineThreads = 256;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Per (loop, tone, dimension, residue): g and g' by one warp summing the M_d aliases.
__global__ void tone_response_kernel(RefineGeom rg, DeviceTables t, const float* __restrict__ freq, int K,
                                     float2* __restrict__ gres, float2* __restrict__ gder) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  const int64_t total = static_cast<int64_t>(rg.loops) * K * rg.sumb;
  for (int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < total; w += warps) {
    const int pos = static_cast<int>(w % rg.sumb);
    const int k = static_cast<int>((w / rg.sumb) % K);
    const int l = static_cast<int>(w / (static_cast<int64_t>(rg.sumb) * K));
    int d = 0;
    while (d + 1 < rg.ndim && pos >= rg.boff[d + 1]) ++d;
    const int x = pos - rg.boff[d];
    float f = freq[k * rg.ndim + d];
    f -= floorf(f);
    // f in [0, 1) as a 64-bit fixed-point phase increment
    const double fd = static_cast<double>(f) * 18446744073709551616.0;
    const uint64_t fx = fd >= 18446744073709551615.0 ? ~0ull : static_cast<uint64_t>(fd);
    const float2* wd = t.wtab[d] + static_cast<int64_t>(l) * rg.n[d];
    float2 acc = make_float2(0.f, 0.f), accd = make_float2(0.f, 0.f);
    for (int64_t m = lane; m < rg.m[d]; m += 32) {
      const int64_t s = x + rg.b[d] * m;
      const uint64_t ph = fx * static_cast<uint64_t>(s);
      const float tt = static_cast<float>(ph >> 40) * 5.9604644775390625e-8f;  // 2^-24
      float sn, cs;
      sincospif(2.f * tt, &sn, &cs);
      const float2 term = cmulf(wd[s], make_float2(cs, sn));
      acc.x += term.x;
      acc.y += term.y;
      const float ws = 6.283185307179586f * static_cast<float>(s);  // j 2 pi s
      accd.x -= ws * term.y;
      accd.y += ws * term.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      accd.x += __shfl_xor_sync(0xffffffffu, accd.x, o);
      accd.y += __shfl_xor_sync(0xffffffffu, accd.y, o);
    }
    if (lane == 0) {
      gres[w] = acc;
      gder[w] = accd;
    }
  }
}

// Residual buckets in source residue order, R_l[x] = F_l[sigma^{-1} x] - sum_k a_k prod_d g,
// and per-block partial sums of |R|^2 (double).
__global__ void __launch_bounds__(kRefineThreads) residual_kernel(RefineGeom rg, DeviceTables t,
                                                                  const float2* __restrict__ folded,
                                                                  const float2* __restrict__ gres,
                                                                  const float2* __restrict__ amp, int K,
                                                                  float2* __restrict__ resid,
                                                                  double* __restrict__ partial) {
  __shared__ double red[kRefineThreads / 32];
  const int64_t total = static_cast<int64_t>(rg.loops) * rg.total_b;
  double local = 0.0;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int l = static_cast<int>(e / rg.total_b);
    const int64_t x = e - static_cast<int64_t>(l) * rg.total_b;
    int xd[kMaxDim];
    int64_t j = 0;
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d) {
      xd[d] = 0;
      if (d < rg.ndim) {
        xd[d] = static_cast<int>((x >> rg.b_shift[d]) & (rg.b[d] - 1));
        const int jd = (t.sigma_inv_b[l * rg.ndim + d] * xd[d]) & static_cast<int>(rg.b[d] - 1);
        j += static_cast<int64_t>(jd) << rg.b_shift[d];
      }
    }
    float2 model = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
      const float2* gk = gres + (static_cast<int64_t>(l) * K + k) * rg.sumb;
      float2 p = amp[k];
#pragma unroll
      for (int d = 0; d < kMaxDim; ++d)
        if (d < rg.ndim) p = cmulf(p, gk[rg.boff[d] + xd[d]]);
      model.x += p.x;
      model.y += p.y;
    }
    const float2 fv = folded[static_cast<int64_t>(l) * rg.total_b + j];
    const float2 r = make_float2(fv.x - model.x, fv.y - model.y);
    resid[e] = r;
    local += static_cast<double>(r.x) * r.x + static_cast<double>(r.y) * r.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kRefineThreads / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

// Contraction layout per (loop, tone), kVals values: [0, 1] S = sum conj(R) J_a, [2] sum |J_a|^2,
// [3 + 2d, 4 + 2d] T_d = sum conj(R) P_d, [11 + d] sum |P_d|^2, [15 + 2d, 16 + 2d] C_d = sum conj(J_a) P_d,
// [23 + 2p, 24 + 2p] Q_p = sum conj(P_d) P_e for the p-th pair d < e, with J_a = prod_d g_d (the
// derivative of the model by the amplitude) and P_d = g'_d prod_{e != d} g_e (by f_d, over a_k).
constexpr int kPairs = kMaxDim * (kMaxDim - 1) / 2;
constexpr int kVals = 3 + 5 * kMaxDim + 2 * kPairs;

__host__ __device__ __forceinline__ int pair_index(int d, int e) {  // d < e
  int p = 0;
  for (int i = 0; i < d; ++i) p += kMaxDim - 1 - i;
  return p + (e - d - 1);
}

// One block per (loop, tone): the sums above over the loop's B buckets.
__global__ void __launch_bounds__(kRefineThreads) contract_kernel(RefineGeom rg, const float2* __restrict__ resid,
                                                                  const float2* __restrict__ gres,
                                                                  const float2* __restrict__ gder, int K,
                                                                  float* __restrict__ out) {
  __shared__ double red[kRefineThreads / 32][kVals];
  const int lk = blockIdx.x;
  const int l = lk / K;
  const float2* gk = gres + static_cast<int64_t>(lk) * rg.sumb;
  const float2* dk = gder + static_cast<int64_t>(lk) * rg.sumb;
  const float2* rl = resid + static_cast<int64_t>(l) * rg.total_b;
  float v[kVals];  // per-thread sums in FP32 (a few dozen terms), the block sum in FP64
#pragma unroll
  for (int i = 0; i < kVals; ++i) v[i] = 0.f;
  for (int64_t x = threadIdx.x; x < rg.total_b; x += blockDim.x) {
    float2 gx[kMaxDim], dx[kMaxDim];
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d) {
      gx[d] = make_float2(1.f, 0.f);
      dx[d] = make_float2(0.f, 0.f);
      if (d < rg.ndim) {
        const int xd = static_cast<int>((x >> rg.b_shift[d]) & (rg.b[d] - 1));
        gx[d] = gk[rg.boff[d] + xd];
        dx[d] = dk[rg.boff[d] + xd];
      }
    }
    const float2 r = rl[x];
    const float2 c = make_float2(r.x, -r.y);  // conj(R)
    float2 ja = make_float2(1.f, 0.f);
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d)
      if (d < rg.ndim) ja = cmulf(ja, gx[d]);
    const float2 cja = make_float2(ja.x, -ja.y);
    const float2 s = cmulf(c, ja);
    v[0] += s.x;
    v[1] += s.y;
    v[2] += ja.x * ja.x + ja.y * ja.y;
    float2 pd[kMaxDim];
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d) {
      pd[d] = make_float2(0.f, 0.f);
      if (d < rg.ndim) {
        float2 q = dx[d];
#pragma unroll
        for (int e = 0; e < kMaxDim; ++e)
          if (e < rg.ndim && e != d) q = cmulf(q, gx[e]);
        pd[d] = q;
        const float2 td = cmulf(c, q);
        v[3 + 2 * d] += td.x;
        v[4 + 2 * d] += td.y;
        v[3 + 2 * kMaxDim + d] += q.x * q.x + q.y * q.y;
        const float2 cd = cmulf(cja, q);
        v[3 + 3 * kMaxDim + 2 * d] += cd.x;
        v[4 + 3 * kMaxDim + 2 * d] += cd.y;
      }
    }
#pragma unroll
    for (int d = 0; d < kMaxDim; ++d)
#pragma unroll
      for (int e = d + 1; e < kMaxDim; ++e)
        if (e < rg.ndim) {
          const float2 q = cmulf(make_float2(pd[d].x, -pd[d].y), pd[e]);
          const int p = pair_index(d, e);
          v[3 + 5 * kMaxDim + 2 * p] += q.x;
          v[4 + 5 * kMaxDim + 2 * p] += q.y;
        }
  }
  double vd[kVals];
#pragma unroll
  for (int i = 0; i < kVals; ++i) {
    vd[i] = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vd[i] += __shfl_xor_sync(0xffffffffu, vd[i], o);
  }
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int i = 0; i < kVals; ++i) red[threadIdx.x >> 5][i] = vd[i];
  __syncthreads();
  if (threadIdx.x < kVals) {
    double t = 0.0;
    for (int w = 0; w < kRefineThreads / 32; ++w) t += red[w][threadIdx.x];
    out[static_cast<int64_t>(lk) * kVals + threadIdx.x] = static_cast<float>(t);
  }
}

// Per tone: sums over loops (fixed order) into the gradient and the Gauss-Newton matrix of the
// real parameters (a_re, a_im, f_0 .. f_{D-1}); thread 0 of block 0 also sums the loss
// partials.  With gh set, each tone's g and H go there ([K][P + P^2], P = D + 2) for the
// Levenberg-Marquardt iteration.
__global__ void finish_kernel(RefineGeom rg, const float* __restrict__ out, int K, const double* __restrict__ partial,
                              int nparts, const float2* __restrict__ amp, double* loss, float* grad_freq,
                              float2* grad_amp, float* hdiag, double* gh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0 && loss) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += partial[i];
    *loss = s;
  }
  if (k >= K) return;
  double acc[kVals];
  for (int i = 0; i < kVals; ++i) acc[i] = 0.0;
  for (int l = 0; l < rg.loops; ++l) {
    const float* o = out + (static_cast<int64_t>(l) * K + k) * kVals;
    for (int i = 0; i < kVals; ++i) acc[i] += o[i];
  }
  const int D = rg.ndim;
  const float2 a = amp[k];
  const double ar = a.x, ai = a.y, a2 = ar * ar + ai * ai;
  // gradient: dE/da_re = -2 Re S, dE/da_im = 2 Im S, dE/df_d = -2 Re(a T_d)
  double g[kMaxDim + 2];
  g[0] = -2.0 * acc[0];
  g[1] = 2.0 * acc[1];
  for (int d = 0; d < D; ++d) g[2 + d] = -2.0 * (ar * acc[3 + 2 * d] - ai * acc[4 + 2 * d]);
  // Gauss-Newton matrix 2 Re sum conj(J_p) J_q of the real parameters
  double H[kMaxDim + 2][kMaxDim + 2];
  const int P = D + 2;
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j) H[i][j] = 0.0;
  H[0][0] = H[1][1] = 2.0 * acc[2];
  for (int d = 0; d < D; ++d) {
    const double cre = acc[3 + 3 * kMaxDim + 2 * d], cim = acc[4 + 3 * kMaxDim + 2 * d];
    const double acr = ar * cre - ai * cim, aci = ar * cim + ai * cre;  // a C_d
    H[0][2 + d] = H[2 + d][0] = 2.0 * acr;
    H[1][2 + d] = H[2 + d][1] = 2.0 * aci;
    H[2 + d][2 + d] = 2.0 * a2 * acc[3 + 2 * kMaxDim + d];
    for (int e = d + 1; e < D; ++e) {
      const double q = 2.0 * a2 * acc[3 + 5 * kMaxDim + 2 * pair_index(d, e)];
      H[2 + d][2 + e] = H[2 + e][2 + d] = q;
    }
  }
  if (grad_amp) grad_amp[k] = make_float2(static_cast<float>(g[0]), static_cast<float>(g[1]));
  for (int d = 0; d < D; ++d) {
    if (grad_freq) grad_freq[k * D + d] = static_cast<float>(g[2 + d]);
    if (hdiag) hdiag[k * (D + 1) + 1 + d] = static_cast<float>(H[2 + d][2 + d]);
  }
  if (hdiag) hdiag[k * (D + 1)] = static_cast<float>(H[0][0]);
  if (gh) {
    double* o = gh + static_cast<int64_t>(k) * kLmTone;
    for (int i = 0; i < P; ++i) o[i] = g[i];
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < P; ++j) o[P + i * P + j] = H[i][j];
  }
}

constexpr double kLambda0 = 1e-3, kLambdaMin = 1e-7, kLambdaMax = 1e7;

// One Levenberg-Marquardt iteration over all tones, with Marquardt's adaptive damping.  The
// tones' current parameters (the trial just evaluated) are accepted when their loss is below
// the accepted point's (always on the first call, iter = 0), and lambda shrinks tenfold;
// otherwise the tones return to the accepted point and lambda grows tenfold.  Each tone then
// solves (H + lambda diag H) delta = -g at the accepted point (FP64, Gaussian elimination with
// pivoting) and moves to accepted + lr delta, the next trial (frequencies wrapped into
// [0, 1)); on the final call it stays at the accepted point instead.  Every thread derives the
// decision and lambda from the same values; thread 0 writes them to the other half of the
// double-buffered state ([2][E, lambda]; state[4] = the trial's loss) for the next call.
__global__ void lm_kernel(RefineGeom rg, int K, float* freq, float2* amp, double* gh, float* acc_freq,
                          float2* acc_amp, double* state, int iter, float lr, int final_call) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const double* prev = state + 2 * (iter & 1);
  const double e_trial = state[4];
  const bool accept = iter == 0 || e_trial < prev[0];  // a NaN loss is never below
  const double lambda = iter == 0 ? kLambda0
                        : accept  ? fmax(prev[1] * 0.1, kLambdaMin)
                                  : fmin(prev[1] * 10.0, kLambdaMax);
  if (k == 0) {
    double* next = state + 2 * ((iter + 1) & 1);
    next[0] = accept ? e_trial : prev[0];
    next[1] = lambda;
  }
  if (k >= K) return;
  const int D = rg.ndim, P = D + 2;
  const double* trial = gh + static_cast<int64_t>(k) * kLmTone;
  double* acc = gh + (static_cast<int64_t>(K) + k) * kLmTone;
  if (accept) {
    for (int i = 0; i < P + P * P; ++i) acc[i] = trial[i];
    for (int d = 0; d < D; ++d) acc_freq[k * D + d] = freq[k * D + d];
    acc_amp[k] = amp[k];
  }
  const float2 a0 = acc_amp[k];
  if (final_call) {
    amp[k] = a0;
    for (int d = 0; d < D; ++d) freq[k * D + d] = acc_freq[k * D + d];
    return;
  }
  double M[kMaxDim + 2][kMaxDim + 3];
  for (int i = 0; i < P; ++i) {
    for (int j = 0; j < P; ++j) M[i][j] = acc[P + i * P + j];
    M[i][i] += lambda * acc[P + i * P + i] + 1e-30;
    M[i][P] = -acc[i];
  }
  bool ok = true;
  for (int c = 0; c < P && ok; ++c) {
    int piv = c;
    for (int r = c + 1; r < P; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (!(fabs(M[piv][c]) > 0.0)) {
      ok = false;
      break;
    }
    if (piv != c)
      for (int j = c; j <= P; ++j) {
        const double tmp = M[c][j];
        M[c][j] = M[piv][j];
        M[piv][j] = tmp;
      }
    for (int r = c + 1; r < P; ++r) {
      const double f = M[r][c] / M[c][c];
      for (int j = c; j <= P; ++j) M[r][j] -= f * M[c][j];
    }
  }
  double delta[kMaxDim + 2];
  for (int i = 0; i < P; ++i) delta[i] = 0.0;
  if (ok)
    for (int i = P - 1; i >= 0; --i) {
      double t = M[i][P];
      for (int j = i + 1; j < P; ++j) t -= M[i][j] * delta[j];
      delta[i] = t / M[i][i];
    }
  amp[k] = make_float2(static_cast<float>(a0.x + lr * delta[0]), static_cast<float>(a0.y + lr * delta[1]));
  for (int d = 0; d < D; ++d) {
    double f = acc_freq[k * D + d] + lr * delta[2 + d];
    f -= floor(f);
    freq[k * D + d] = static_cast<float>(f);
  }
}

}  // namespace

cudaError_t launch_refine_eval(const RefineGeom& rg, const DeviceTables& t, const RefineWork& w,
                               const float2* folded, int K, const float* freq, const float2* amp, double* loss,
                               float* grad_freq, float2* grad_amp, float* hdiag, double* gh, cudaStream_t stream) {
  const int64_t warps = static_cast<int64_t>(rg.loops) * K * rg.sumb;
  int blocks = static_cast<int>(std::min<int64_t>((warps + 7) / 8, 152 * 16));
  tone_response_kernel<<<std::max(blocks, 1), 256, 0, stream>>>(rg, t, freq, K, w.gres, w.gder);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  residual_kernel<<<w.parts, kRefineThreads, 0, stream>>>(rg, t, folded, w.gres, amp, K, w.resid, w.partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  contract_kernel<<<rg.loops * K, kRefineThreads, 0, stream>>>(rg, w.resid, w.gres, w.gder, K, w.contr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  finish_kernel<<<(K + 127) / 128, 128, 0, stream>>>(rg, w.contr, K, w.partial, w.parts, amp, loss, grad_freq,
                                                     grad_amp, hdiag, gh);
  return cudaGetLastError();
}

cudaError_t launch_refine_step(const RefineGeom& rg, const DeviceTables& t, const RefineWork& w,
                               const float2* folded, int K, float* freq, float2* amp, int iter, float lr,
                               bool final_call, cudaStream_t stream) {
  cudaError_t e = launch_refine_eval(rg, t, w, folded, K, freq, amp, w.lm_state + 4, nullptr, nullptr, nullptr,
                                     w.lm_gh, stream);
  if (e != cudaSuccess) return e;
  lm_kernel<<<(K + 127) / 128, 128, 0, stream>>>(rg, K, freq, amp, w.lm_gh, w.lm_freq, w.lm_amp, w.lm_state, iter,
                                                 lr, final_call ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace rsft
