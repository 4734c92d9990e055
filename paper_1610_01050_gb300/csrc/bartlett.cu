// Dense comparison detector: the Bartlett method of Appendix A (Algorithm 2) with one
// data segment.  The cube is windowed by the product of the per-dimension pre-windows
// (§III-C), transformed by the full N-point N-D FFT (cuFFT, forward, unnormalised) and
// each bin's power is compared with the exact one-segment Neyman-Pearson threshold
// gamma = -sigma_n^2 ||w||^2 ln P_fa (the H0 bin power is exponential with mean
// sigma_n^2 ||w||^2).  Detections come out in ascending row-major order: a count pass
// gives the hits of each range of kRange bins, a scan turns them into offsets, and a
// write pass emits each range's hits in order (warp ballots), with the amplitude
// u-hat_k / prod_d sum_t w_d(t).
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <string>
#include <vector>

#include "device.cuh"
#include "plan_host.h"
#include "rsft.h"

namespace rsft {
namespace {

constexpr int kRange = 2048;  // bins per warp range of the detection passes

struct DenseGeom {
  int ndim;
  int64_t n[kMaxDim];
  int log_n[kMaxDim];
  int woff[kMaxDim];  // offset of w_d in the concatenated window table
  int64_t total;
};

// u(s) = r(s) prod_d w_d(s_d): one complex element per thread.
__global__ void window_kernel(const float2* __restrict__ x, float2* __restrict__ u, const float* __restrict__ w,
                              DenseGeom g) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < g.total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint64_t r = static_cast<uint64_t>(e);
    float wv = 1.f;
#pragma unroll
    for (int d = kMaxDim - 1; d >= 0; --d) {
      if (d < g.ndim) {
        wv *= __ldg(w + g.woff[d] + static_cast<int>(r & static_cast<uint64_t>(g.n[d] - 1)));
        r >>= g.log_n[d];
      }
    }
    const float2 v = x[e];
    u[e] = make_float2(v.x * wv, v.y * wv);
  }
}

// Hits (|u-hat_k|^2 > gamma) of each range of kRange bins, one warp per range.
__global__ void dense_count_kernel(const float2* __restrict__ spec, int64_t total, float gamma,
                                   uint32_t* __restrict__ range_count, int64_t ranges) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t rg = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; rg < ranges; rg += warps) {
    const int64_t base = rg * kRange;
    uint32_t cnt = 0;
    for (int i = lane; i < kRange; i += 32) {
      const int64_t k = base + i;
      if (k < total) {
        const float2 v = spec[k];
        cnt += (v.x * v.x + v.y * v.y > gamma) ? 1u : 0u;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) range_count[rg] = cnt;
  }
}

// Ordered write of each range's hits from its scanned offset.
__global__ void dense_write_kernel(const float2* __restrict__ spec, int64_t total, float gamma,
                                   const uint64_t* __restrict__ range_off, int64_t ranges, float inv_gain,
                                   uint64_t* __restrict__ located, float2* __restrict__ amp, int64_t capacity) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
  for (int64_t rg = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; rg < ranges; rg += warps) {
    const int64_t base = rg * kRange;
    uint64_t pos = range_off[rg];
    if (range_off[rg + 1] == pos) continue;  // no hits in this range
    for (int i0 = 0; i0 < kRange; i0 += 32) {
      const int64_t k = base + i0 + lane;
      float2 v = make_float2(0.f, 0.f);
      bool hit = false;
      if (k < total) {
        v = spec[k];
        hit = v.x * v.x + v.y * v.y > gamma;
      }
      const unsigned bal = __ballot_sync(0xffffffffu, hit);
      if (hit) {
        const uint64_t out = pos + static_cast<uint64_t>(__popc(bal & ((1u << lane) - 1u)));
        if (out < static_cast<uint64_t>(capacity)) {
          located[out] = static_cast<uint64_t>(k);
          if (amp) amp[out] = make_float2(v.x * inv_gain, v.y * inv_gain);
        }
      }
      pos += static_cast<uint64_t>(__popc(bal));
    }
  }
}

}  // namespace
}  // namespace rsft

struct rsft_bartlett_plan {
  int device = 0;
  int64_t max_located = 0;
  rsft::DenseGeom geom{};
  std::vector<double> windows;  // concatenated w_d
  double gamma = 0.0, gain = 0.0;
  float* d_w = nullptr;
  float2* d_spec = nullptr;
  uint32_t* d_range_count = nullptr;
  uint64_t* d_range_off = nullptr;
  int64_t ranges = 0;
  int64_t* d_count = nullptr;
  int64_t* h_count = nullptr;
  cufftHandle fft_a = 0, fft_b = 0;
  bool has_a = false, has_b = false;
  size_t fft_work = 0;
};

namespace {

rsft_status bfail(rsft_status st, const std::string& msg) {
  rsft::set_last_error(msg.c_str());
  return st;
}

rsft_status bcuda(cudaError_t e, const char* where) {
  return bfail(RSFT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

rsft_status bfft(cufftResult r, const char* where) {
  return bfail(RSFT_ERR_CUDA, std::string(where) + ": cuFFT error " + std::to_string(static_cast<int>(r)));
}

struct BDeviceGuard {
  int prev = -1;
  explicit BDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~BDeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void release(rsft_bartlett_plan* p) {
  if (p->has_a) cufftDestroy(p->fft_a);
  if (p->has_b) cufftDestroy(p->fft_b);
  cudaFree(p->d_w);
  cudaFree(p->d_spec);
  cudaFree(p->d_range_count);
  cudaFree(p->d_range_off);
  cudaFree(p->d_count);
  if (p->h_count) cudaFreeHost(p->h_count);
}

rsft_status run_dense(rsft_bartlett_plan* p, const void* d_cube, cudaStream_t s, uint64_t* d_located, void* d_amp,
                      int64_t* d_count) {
  const rsft::DenseGeom& g = p->geom;
  if (reinterpret_cast<uintptr_t>(d_cube) % 16 != 0) return bfail(RSFT_ERR_INVALID_ARG, "cube must be 16-byte aligned");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const int blocks = std::max(1, sms) * 8;
  rsft::window_kernel<<<blocks, 256, 0, s>>>(static_cast<const float2*>(d_cube), p->d_spec, p->d_w, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(e, "dense window");
  cufftResult r = cufftSetStream(p->fft_a, s);
  if (r == CUFFT_SUCCESS) r = cufftExecC2C(p->fft_a, reinterpret_cast<cufftComplex*>(p->d_spec),
                                           reinterpret_cast<cufftComplex*>(p->d_spec), CUFFT_FORWARD);
  if (r == CUFFT_SUCCESS && p->has_b) {
    r = cufftSetStream(p->fft_b, s);
    if (r == CUFFT_SUCCESS) r = cufftExecC2C(p->fft_b, reinterpret_cast<cufftComplex*>(p->d_spec),
                                             reinterpret_cast<cufftComplex*>(p->d_spec), CUFFT_FORWARD);
  }
  if (r != CUFFT_SUCCESS) return bfft(r, "dense N-D FFT");
  const float gamma = static_cast<float>(p->gamma);
  rsft::dense_count_kernel<<<blocks, 256, 0, s>>>(p->d_spec, g.total, gamma, p->d_range_count, p->ranges);
  if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(e, "dense count");
  if ((e = rsft::launch_count_scan(p->d_range_count, p->ranges, p->d_range_off, d_count, s)) != cudaSuccess)
    return bcuda(e, "dense scan");
  rsft::dense_write_kernel<<<blocks, 256, 0, s>>>(p->d_spec, g.total, gamma, p->d_range_off, p->ranges,
                                                  static_cast<float>(1.0 / p->gain), d_located,
                                                  static_cast<float2*>(d_amp), p->max_located);
  if ((e = cudaGetLastError()) != cudaSuccess) return bcuda(e, "dense write");
  return RSFT_OK;
}

}  // namespace

extern "C" rsft_status rsft_bartlett_plan_create(const rsft_desc* desc, rsft_bartlett_plan** plan) {
  if (!desc || !plan) return bfail(RSFT_ERR_INVALID_ARG, "NULL descriptor or plan");
  *plan = nullptr;
  if (desc->ndim < 1 || desc->ndim > 4) return bfail(RSFT_ERR_INVALID_ARG, "ndim must be 1..4");
  if (!(desc->p_fa > 0.0 && desc->p_fa < 1.0)) return bfail(RSFT_ERR_INVALID_ARG, "p_fa must lie in (0, 1)");
  if (!(desc->noise_var > 0.0)) return bfail(RSFT_ERR_INVALID_ARG, "noise_var must be positive");
  if (desc->max_located < 0) return bfail(RSFT_ERR_INVALID_ARG, "max_located must be >= 0");
  if (desc->window != RSFT_WIN_CHEB && desc->window != RSFT_WIN_RECT) return bfail(RSFT_ERR_INVALID_ARG, "unknown window");
  rsft_bartlett_plan* p = new rsft_bartlett_plan();
  p->device = desc->device < 0 ? 0 : desc->device;
  p->max_located = desc->max_located;
  rsft::DenseGeom& g = p->geom;
  g.ndim = desc->ndim;
  g.total = 1;
  double energy = 1.0, gain = 1.0;
  int off = 0;
  for (int d = 0; d < rsft::kMaxDim; ++d) {
    g.n[d] = 1;
    g.log_n[d] = 0;
    g.woff[d] = 0;
  }
  for (int d = 0; d < g.ndim; ++d) {
    const int64_t n = desc->n[d];
    if (n < 1 || (n & (n - 1)) != 0) {
      delete p;
      return bfail(RSFT_ERR_INVALID_ARG, "n_d must be a power of two");
    }
    g.n[d] = n;
    while ((int64_t(1) << g.log_n[d]) < n) ++g.log_n[d];
    g.woff[d] = off;
    std::vector<double> w = desc->window == RSFT_WIN_RECT ? std::vector<double>(n, 1.0)
                                                          : rsft::chebyshev_window(n, desc->atten_db);
    double e2 = 0.0, s1 = 0.0;
    for (double v : w) {
      e2 += v * v;
      s1 += v;
    }
    energy *= e2;
    gain *= s1;
    p->windows.insert(p->windows.end(), w.begin(), w.end());
    off += static_cast<int>(n);
    g.total *= n;
  }
  if (g.total > 0x7fffffffll) {
    delete p;
    return bfail(RSFT_ERR_UNSUPPORTED, "more than 2^31 - 1 points");
  }
  p->gamma = -desc->noise_var * energy * std::log(desc->p_fa);
  p->gain = gain;
  p->ranges = (g.total + rsft::kRange - 1) / rsft::kRange;
  BDeviceGuard guard(p->device);
  std::vector<float> wf(p->windows.begin(), p->windows.end());
  cudaError_t e = cudaMalloc(&p->d_w, wf.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(p->d_w, wf.data(), wf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_spec, static_cast<size_t>(g.total) * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&p->d_range_count, static_cast<size_t>(p->ranges) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_range_off, static_cast<size_t>(p->ranges + 1) * 8);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_count, 16);
  if (e == cudaSuccess) e = cudaMallocHost(&p->h_count, 16);
  if (e != cudaSuccess) {
    release(p);
    delete p;
    return e == cudaErrorMemoryAllocation ? bfail(RSFT_ERR_OOM, "dense plan allocation") : bcuda(e, "dense plan");
  }
  // cuFFT: one plan of rank ndim (<= 3), or for 4-D a rank-3 plan over the last three
  // dimensions (batched over the first) and a strided 1-D plan over the first
  int dims[3];
  cufftResult r;
  if (g.ndim <= 3) {
    for (int d = 0; d < g.ndim; ++d) dims[d] = static_cast<int>(g.n[d]);
    r = cufftPlanMany(&p->fft_a, g.ndim, dims, nullptr, 1, 0, nullptr, 1, 0, CUFFT_C2C, 1);
    p->has_a = r == CUFFT_SUCCESS;
  } else {
    for (int d = 0; d < 3; ++d) dims[d] = static_cast<int>(g.n[d + 1]);
    const int inner = static_cast<int>(g.n[1] * g.n[2] * g.n[3]);
    r = cufftPlanMany(&p->fft_a, 3, dims, nullptr, 1, inner, nullptr, 1, inner, CUFFT_C2C, static_cast<int>(g.n[0]));
    p->has_a = r == CUFFT_SUCCESS;
    if (r == CUFFT_SUCCESS) {
      int n0 = static_cast<int>(g.n[0]);
      r = cufftPlanMany(&p->fft_b, 1, &n0, &n0, inner, 1, &n0, inner, 1, CUFFT_C2C, inner);
      p->has_b = r == CUFFT_SUCCESS;
    }
  }
  if (r != CUFFT_SUCCESS) {
    release(p);
    delete p;
    return bfft(r, "cuFFT plan");
  }
  size_t wa = 0, wb = 0;
  cufftGetSize(p->fft_a, &wa);
  if (p->has_b) cufftGetSize(p->fft_b, &wb);
  p->fft_work = wa + wb;
  *plan = p;
  return RSFT_OK;
}

extern "C" void rsft_bartlett_plan_destroy(rsft_bartlett_plan* plan) {
  if (!plan) return;
  BDeviceGuard guard(plan->device);
  release(plan);
  delete plan;
}

extern "C" rsft_status rsft_bartlett_execute_async(rsft_bartlett_plan* plan, const void* d_cube, void* stream,
                                                   uint64_t* d_located, void* d_amp, int64_t* d_n_located) {
  if (!plan || !d_cube || !d_n_located) return bfail(RSFT_ERR_INVALID_ARG, "NULL plan, cube or count");
  if (plan->max_located > 0 && !d_located) return bfail(RSFT_ERR_INVALID_ARG, "d_located is NULL");
  BDeviceGuard guard(plan->device);
  return run_dense(plan, d_cube, static_cast<cudaStream_t>(stream), d_located, d_amp, d_n_located);
}

extern "C" rsft_status rsft_bartlett_execute(rsft_bartlett_plan* plan, const void* d_cube, void* stream,
                                             uint64_t* d_located, void* d_amp, int64_t* n_located) {
  if (!plan || !d_cube || !n_located) return bfail(RSFT_ERR_INVALID_ARG, "NULL plan, cube or count");
  if (plan->max_located > 0 && !d_located) return bfail(RSFT_ERR_INVALID_ARG, "d_located is NULL");
  BDeviceGuard guard(plan->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rsft_status st = run_dense(plan, d_cube, s, d_located, d_amp, plan->d_count);
  if (st != RSFT_OK) return st;
  cudaError_t e = cudaMemcpyAsync(plan->h_count, plan->d_count, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bcuda(e, "rsft_bartlett_execute");
  *n_located = plan->h_count[0];
  if (*n_located > plan->max_located) return bfail(RSFT_ERR_CAPACITY, "located list truncated to max_located");
  return RSFT_OK;
}

extern "C" rsft_status rsft_bartlett_get(const rsft_bartlett_plan* plan, int32_t what, void* out, size_t bytes) {
  if (!plan || !out) return bfail(RSFT_ERR_INVALID_ARG, "NULL plan or output");
  switch (what) {
    case RSFT_BARTLETT_GAMMA:
      if (bytes < 8) break;
      *static_cast<double*>(out) = plan->gamma;
      return RSFT_OK;
    case RSFT_BARTLETT_GAIN:
      if (bytes < 8) break;
      *static_cast<double*>(out) = plan->gain;
      return RSFT_OK;
    case RSFT_BARTLETT_WINDOW:
      if (bytes < plan->windows.size() * 8) break;
      for (size_t i = 0; i < plan->windows.size(); ++i) static_cast<double*>(out)[i] = plan->windows[i];
      return RSFT_OK;
    case RSFT_BARTLETT_WORKSPACE_BYTES:
      if (bytes < 8) break;
      *static_cast<int64_t*>(out) = static_cast<int64_t>(plan->geom.total * 8 + plan->ranges * 12 + plan->fft_work);
      return RSFT_OK;
    default:
      return bfail(RSFT_ERR_INVALID_ARG, "unknown rsft_bartlett_get item");
  }
  return bfail(RSFT_ERR_INVALID_ARG, "output buffer too small");
}

extern "C" rsft_status rsft_bartlett_copy_spectrum(const rsft_bartlett_plan* plan, void* d_out, void* stream) {
  if (!plan || !d_out) return bfail(RSFT_ERR_INVALID_ARG, "NULL plan or output");
  BDeviceGuard guard(plan->device);
  cudaError_t e = cudaMemcpyAsync(d_out, plan->d_spec, static_cast<size_t>(plan->geom.total) * 8,
                                  cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RSFT_OK : bcuda(e, "rsft_bartlett_copy_spectrum");
}
