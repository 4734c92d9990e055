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
// A CTA owns one residue class of the row dimensions, a chunk of that class's
// rows, and a chunk of W columns; each thread keeps two fixed adjacent columns
// and walks the rows, so its column weights factor out of the row loop:
//     acc_l(c) = sum_rows a_l^{row}(row) r(row, c),   contribution a_l^{col}(c) acc_l(c).
// Row weights for all loops of the group sit in shared memory as
// (re, re, -im, im) so one complex multiply-add is two packed FP32x2 FMAs.
// Sums over threads use a fixed order (deterministic results).
#include "device.cuh"

namespace rsft {
namespace {

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct FoldArgs {
  const float4* cube;
  Geometry g;
  FoldSchedule fs;
  DeviceTables t;
  int loop0;
  int log_width;
  float2* folded;
  float2* partial;
};

constexpr int kUnroll = 4;

template <int LG>
__global__ void __launch_bounds__(kFoldThreads, 2) fold_kernel(const FoldArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  const FoldSchedule& fs = a.fs;
  const int tid = threadIdx.x;
  const int chunks = fs.row_chunks * fs.col_chunks;
  const int cc = blockIdx.x % fs.col_chunks;
  const int rc = (blockIdx.x / fs.col_chunks) % fs.row_chunks;
  const int cls = blockIdx.x / chunks;
  const int R = fs.rows_per_chunk;

  // residues of the row dimensions for this class (row-major over [0, d_in))
  int xo[kMaxDim];
  {
    int c = cls;
#pragma unroll
    for (int e = kMaxDim - 1; e >= 0; --e) {
      xo[e] = 0;
      if (e < fs.d_in) {
        xo[e] = c & static_cast<int>(g.b[e] - 1);
        c >>= g.log_b[e];
      }
    }
  }

  // ---- row table: global row index and (re, re, -im, im) row weight per loop
  float4* wrow = reinterpret_cast<float4*>(smem);
  uint32_t* rowidx = reinterpret_cast<uint32_t*>(smem + static_cast<size_t>(R) * LG * sizeof(float4));
  for (int e = tid; e < R * LG; e += kFoldThreads) {
    const int rl = e / LG;
    const int l = e - rl * LG;
    int r = rc * R + rl;
    float2 w = make_float2(1.f, 0.f);
    uint32_t row = 0, stride = 1;
#pragma unroll
    for (int d = kMaxDim - 1; d >= 0; --d) {
      if (d < fs.d_in) {
        const int mdig = r & static_cast<int>(g.m[d] - 1);
        r >>= g.log_m[d];
        const uint32_t s = static_cast<uint32_t>(xo[d]) + (static_cast<uint32_t>(mdig) << g.log_b[d]);
        row += s * stride;
        stride *= static_cast<uint32_t>(g.n[d]);
        w = cmul(w, __ldg(a.t.wtab[d] + static_cast<int64_t>(a.loop0 + l) * g.n[d] + s));
      }
    }
    wrow[e] = make_float4(w.x, w.x, -w.y, w.y);
    if (l == 0) rowidx[rl] = row;
  }
  __syncthreads();

  // ---- stream the rows: each thread holds columns cp, cp + 1 of the chunk
  const int W = fs.width;
  const int cp = (2 * tid) & (W - 1);
  const int ro = (2 * tid) >> a.log_width;
  const int RS = (2 * kFoldThreads) >> a.log_width;
  const int64_t col = static_cast<int64_t>(cc) * W + cp;
  unsigned long long acc0[LG], acc1[LG];
#pragma unroll
  for (int l = 0; l < LG; ++l) {
    acc0[l] = 0ull;
    acc1[l] = 0ull;
  }
  for (int rl = ro; rl < R; rl += RS * kUnroll) {
    float4 v[kUnroll];
    int rr[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int r2 = rl + u * RS;
      rr[u] = r2 < R ? r2 : 0;
      if (r2 < R) {
        const int64_t off = static_cast<int64_t>(rowidx[r2]) * fs.row_len + col;
        v[u] = __ldcs(a.cube + (off >> 1));
      } else {
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const unsigned long long d0 = pack2(v[u].x, v[u].y), d0s = pack2(v[u].y, v[u].x);
      const unsigned long long d1 = pack2(v[u].z, v[u].w), d1s = pack2(v[u].w, v[u].z);
      const float4* wr = wrow + rr[u] * LG;
#pragma unroll
      for (int l = 0; l < LG; ++l) {
        const float4 w = wr[l];
        const unsigned long long wa = pack2(w.x, w.y), wb = pack2(w.z, w.w);
        acc0[l] = fma2(wa, d0, acc0[l]);
        acc0[l] = fma2(wb, d0s, acc0[l]);
        acc1[l] = fma2(wa, d1, acc1[l]);
        acc1[l] = fma2(wb, d1s, acc1[l]);
      }
    }
  }
  __syncthreads();  // the row table is dead; its space now holds per-thread sums

  // ---- column weights, then a fixed-order reduction over threads of equal residue
  float2* S = reinterpret_cast<float2*>(smem);  // [LG][2 * threads]
  {
    int s0[kMaxDim];
    int64_t c = col;
#pragma unroll
    for (int d = kMaxDim - 1; d >= 0; --d) {
      s0[d] = 0;
      if (d >= fs.d_in && d < g.ndim) {
        s0[d] = static_cast<int>(c & (g.n[d] - 1));
        c >>= g.log_n[d];
      }
    }
    const int last = g.ndim - 1;
#pragma unroll
    for (int l = 0; l < LG; ++l) {
      float2 w0 = make_float2(1.f, 0.f), w1;
#pragma unroll
      for (int d = 0; d < kMaxDim; ++d) {
        if (d >= fs.d_in && d < last) w0 = cmul(w0, __ldg(a.t.wtab[d] + static_cast<int64_t>(a.loop0 + l) * g.n[d] + s0[d]));
      }
      const float2* wl = a.t.wtab[last] + static_cast<int64_t>(a.loop0 + l) * g.n[last];
      w1 = cmul(w0, __ldg(wl + s0[last] + 1));
      w0 = cmul(w0, __ldg(wl + s0[last]));
      S[l * 2 * kFoldThreads + 2 * tid] = cmul(w0, unpack2(acc0[l]));
      S[l * 2 * kFoldThreads + 2 * tid + 1] = cmul(w1, unpack2(acc1[l]));
    }
  }
  __syncthreads();

  const int X = fs.xcount;
  for (int o = tid; o < LG * X; o += kFoldThreads) {
    const int l = o / X;
    const int x = o - l * X;
    float2 sum = make_float2(0.f, 0.f);
    const float2* Sl = S + l * 2 * kFoldThreads;
    for (int k = 0; k < fs.mult; ++k) {
      const int c = a.t.cols_by_x[x * fs.mult + k];
      for (int r = 0; r < RS; ++r) {
        const float2 v = Sl[r * W + c];
        sum.x += v.x;
        sum.y += v.y;
      }
    }
    if (fs.direct) {
      // bucket j = sigma^{-1} x mod B per dimension (paper order)
      const int lg = a.loop0 + l;
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
    } else {
      const int ch = rc * fs.col_chunks + cc;
      a.partial[((static_cast<int64_t>(l) * fs.classes + cls) * chunks + ch) * X + x] = sum;
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

template <int LG>
cudaError_t launch_fold_lg(const FoldArgs& args, int ctas, int smem, cudaStream_t stream) {
  // raise the dynamic shared-memory cap of this instance once per device
  static int configured_smem[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (smem > 48 * 1024 && (dev >= 64 || smem > configured_smem[dev])) {
    e = cudaFuncSetAttribute(fold_kernel<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) configured_smem[dev] = smem;
  }
  fold_kernel<LG><<<ctas, kFoldThreads, smem, stream>>>(args);
  return cudaGetLastError();
}

}  // namespace

int fold_smem_bytes(const FoldSchedule& fs, int lg) {
  const int table = fs.rows_per_chunk * (lg * 16 + 4);
  const int sums = lg * 2 * kFoldThreads * 8;
  return table > sums ? table : sums;
}

cudaError_t launch_fold(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t,
                        const float2* cube, int loop0, int lg, float2* folded, float2* partial,
                        cudaStream_t stream) {
  FoldArgs args;
  args.cube = reinterpret_cast<const float4*>(cube);
  args.g = g;
  args.fs = fs;
  args.t = t;
  args.loop0 = loop0;
  int lw = 0;
  while ((1 << lw) < fs.width) ++lw;
  args.log_width = lw;
  args.folded = folded;
  args.partial = partial;
  const int ctas = fs.classes * fs.row_chunks * fs.col_chunks;
  const int smem = fold_smem_bytes(fs, lg);
  switch (lg) {
    case 1: return launch_fold_lg<1>(args, ctas, smem, stream);
    case 2: return launch_fold_lg<2>(args, ctas, smem, stream);
    case 3: return launch_fold_lg<3>(args, ctas, smem, stream);
    case 4: return launch_fold_lg<4>(args, ctas, smem, stream);
    case 5: return launch_fold_lg<5>(args, ctas, smem, stream);
    case 6: return launch_fold_lg<6>(args, ctas, smem, stream);
    case 7: return launch_fold_lg<7>(args, ctas, smem, stream);
    case 8: return launch_fold_lg<8>(args, ctas, smem, stream);
    case 9: return launch_fold_lg<9>(args, ctas, smem, stream);
    case 10: return launch_fold_lg<10>(args, ctas, smem, stream);
    case 11: return launch_fold_lg<11>(args, ctas, smem, stream);
    case 12: return launch_fold_lg<12>(args, ctas, smem, stream);
    case 13: return launch_fold_lg<13>(args, ctas, smem, stream);
    case 14: return launch_fold_lg<14>(args, ctas, smem, stream);
    case 15: return launch_fold_lg<15>(args, ctas, smem, stream);
    case 16: return launch_fold_lg<16>(args, ctas, smem, stream);
    default: return cudaErrorInvalidValue;
  }
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
