// C ABI of the RSFT hot path (include/rsft.h): plan lifetime, device tables,
// workspace, and the stream-ordered launch sequence of one execute:
//   permute_window_fold (per loop group) -> bucket_fft passes with np_detect in
//   the last pass -> vote_scatter -> stage2_compact -> median_estimate.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "device.cuh"
#include "fold_schedule.h"
#include "plan_host.h"
#include "rsft.h"

using rsft::cplx;

// An extra execution lane of a plan: its own workspace, count block and stream, so
// frames of a batch run concurrently (lane 0 is the plan's own workspace).
struct rsft_lane {
  rsft::Workspace ws{};
  int64_t* d_count = nullptr;   // count, error flag
  int64_t* h_count = nullptr;   // pinned mirror
  bool votes_dirty = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void* staging = nullptr;      // host batches: this lane's cube buffer
  uint64_t* d_loc_stage = nullptr;
  float2* d_amp_stage = nullptr;
};

// Workspace of rsft_execute_frames: the per-frame arrays of up to kMaxFrames frames, one
// frame after another (grown on first use, kept by the plan).
struct rsft_frame_work {
  int cap = 0;                   // frames it holds
  int64_t frame_bits = 0;        // detection words per frame (L * words_b rounded up to whole 16 bytes)
  float2* folded = nullptr;      // [frame][L][B]
  float2* spectrum = nullptr;    // [frame][L][B]
  uint32_t* det_bits = nullptr;  // [frame][frame_bits]
  uint32_t* det_count = nullptr; // [frame][L]
  float* gamma_used = nullptr;   // [frame][L] (estimate mode)
  uint32_t* warp_count = nullptr;
  uint32_t* warp_rows = nullptr;
  ulonglong2* row_list = nullptr;
};

struct rsft_plan {
  rsft::HostPlan host;
  bool has_device = false;
  int device = -1;
  rsft::Geometry geom{};
  rsft::FoldSchedule fold{};
  rsft::VoteRowSchedule rows{};
  bool rows_mode = false;
  std::vector<rsft::FftPass> passes;
  rsft::DeviceTables tables{};
  rsft::Workspace ws{};
  std::vector<void*> allocations;
  std::vector<rsft_lane> lanes;     // extra lanes of batched executes (created on demand)
  rsft::RefineWork refine{};         // bucket-domain refinement scratch (grown on demand)
  rsft::RefineGeom refine_geom{};
  rsft::DeviceTables seg_tables{};  // segment mode: fold tables grouped one loop per launch
  bool seg_ready = false;
  cudaEvent_t fork = nullptr;       // batch fork point on the caller's stream
  int64_t* d_count = nullptr;       // located count of the last execute
  int64_t* h_count = nullptr;       // pinned mirror of d_count
  void* staging = nullptr;          // cube staging buffer of rsft_execute_host
  uint64_t* d_loc_stage = nullptr;  // located list staging of rsft_execute_host
  float2* d_amp_stage = nullptr;
  bool votes_dirty = false;
  bool snr_cached = false;
  double snr_db = 0.0;
  bool timing = false;
  int fold_copy_mode = -1;          // last fold launch: 0 per-row bulk copies, 3/5 tensor box rank,
                                    // 100 + rank on the tensor cores
  bool fold_tc = false;             // the fold runs on the tensor cores (fold_tc.cu)
  bool fft_cluster = false;         // the bucket FFT runs as one cluster launch (else shared-memory passes)
  int fft_csize = 0;                // its CTAs per loop and threads per CTA (0: the default shape; set by
  int fft_threads = 0;              // rsft_plan_autotune)
  rsft_frame_work frames{};         // rsft_execute_frames workspace
  int64_t partial_cap = 0;          // elements of every workspace's fold partial-sum buffer
  int loop_group = rsft::kMaxLoopGroup;  // loops folded per pass over the cube
  int sms = 152;                    // streaming multiprocessors of the plan's device (schedule balance)
  std::vector<int> h_sinvb;                 // [L][D] sigma^{-1} mod B_d (fold kernel parameters)
  std::vector<unsigned short> h_slots, h_xdig;
  std::vector<unsigned char> h_xres;        // residue index of each column of a 64-column chunk
  std::vector<cudaEvent_t> event_pool;
  std::vector<std::array<cudaEvent_t, 6>> pending;  // events of timed executes not yet summed
  struct FramesTiming {
    cudaEvent_t start, end;
    int frames;
  };
  std::vector<FramesTiming> frames_pending;         // fold launches of timed rsft_execute_frames calls
  double frames_fold_ms = 0.0;                      // summed device time of those fold launches
  double frames_folded = 0.0;                       // frames they folded
  double frames_fold_launches = 0.0;
  double stage_ms[6] = {0, 0, 0, 0, 0, 0};
  int64_t timed_executes = 0;
};

namespace {

thread_local std::string g_last_error;

rsft_status fail(rsft_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

rsft_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return RSFT_ERR_CUDA;
}

int ilog2(int64_t v) {
  int r = 0;
  while ((int64_t(1) << r) < v) ++r;
  return r;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <class T>
rsft_status dev_alloc(rsft_plan* p, T** ptr, size_t bytes) {
  void* raw = nullptr;
  cudaError_t e = cudaMalloc(&raw, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? RSFT_ERR_OOM : RSFT_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  p->allocations.push_back(raw);
  *ptr = static_cast<T*>(raw);
  return RSFT_OK;
}

template <class T>
rsft_status upload(rsft_plan* p, T** dst, const std::vector<T>& src) {
  rsft_status st = dev_alloc(p, dst, src.size() * sizeof(T));
  if (st != RSFT_OK) return st;
  cudaError_t e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "upload");
  return RSFT_OK;
}

float2 to_f2(cplx v) { return make_float2(static_cast<float>(v.real()), static_cast<float>(v.imag())); }

// Rows of the vote count: the fewest trailing dimensions whose product of N_d reaches a
// useful row length, bounded by the per-warp shared-memory counters (16 KiB).
bool choose_vote_rows(const rsft::Geometry& g, rsft::VoteRowSchedule& vs) {
  // rows of at most 64 locations use the bit-sliced kernel: the most trailing dimensions that fit
  {
    int best = -1;
    int64_t n_in = 1, b_in = 1, m_in = 1;
    for (int d_v = g.ndim - 1; d_v >= 0; --d_v) {
      n_in *= g.n[d_v];
      b_in *= g.b[d_v];
      m_in *= g.m[d_v];
      if (n_in > 64 || b_in > 64) break;
      best = d_v;
      vs.d_v = d_v;
      vs.n_in = n_in;
      vs.b_in = static_cast<int>(b_in);
      vs.m_in = static_cast<int>(m_in);
    }
    // the kernel keeps a [L][N_d] bucket-offset table (u16) of each row dimension in shared memory
    int64_t kb_words = 0;
    for (int d = 0; best >= 0 && d < vs.d_v; ++d) kb_words += static_cast<int64_t>((g.loops + 7) & ~7) * g.n[d];
    if (best >= 0 && vs.n_in >= 16 && kb_words <= 49152 && g.total_b <= 65536 &&
        rsft::vote_rows_small_smem(g, vs, (g.total_b + 31) / 32) <= 200 * 1024) {
      vs.small = 1;
      vs.rows = g.total_n / vs.n_in;
      vs.rows_per_warp = 64;
      vs.warps = (vs.rows + vs.rows_per_warp - 1) / vs.rows_per_warp;
      return true;
    }
    vs = rsft::VoteRowSchedule{};
  }
  for (int d_v = g.ndim - 1; d_v >= 0; --d_v) {
    int64_t n_in = 1, b_in = 1, m_in = 1;
    for (int e = d_v; e < g.ndim; ++e) {
      n_in *= g.n[e];
      b_in *= g.b[e];
      m_in *= g.m[e];
    }
    if (n_in > 16384 || b_in > 1024) break;
    vs.d_v = d_v;
    vs.n_in = n_in;
    vs.b_in = static_cast<int>(b_in);
    vs.m_in = static_cast<int>(m_in);
    if (n_in >= 64 && (d_v == 0 || n_in * g.n[d_v - 1] > 4096)) break;
  }
  if (vs.n_in == 0 || vs.n_in > 16384 || vs.b_in > 1024) return false;
  vs.rows = g.total_n / vs.n_in;
  int64_t rpw = 4096 / vs.n_in;
  if (rpw < 1) rpw = 1;
  if (rpw > 64) rpw = 64;
  vs.rows_per_warp = static_cast<int>(rpw);
  vs.warps = (vs.rows + rpw - 1) / rpw;
  return true;
}

// Group the bucket dimensions into shared-memory FFT passes, last dimension last.
bool plan_fft_passes(const rsft::Geometry& g, std::vector<rsft::FftPass>& passes) {
  // slab size: about four CTAs per SM over all loops, between 256 and 2048 buckets
  int64_t target = 256;
  while (target < 2048 && target * 4 * 152 < static_cast<int64_t>(g.loops) * g.total_b) target *= 2;
  const int64_t cap = 16384;
  passes.clear();
  int db = g.ndim;
  while (db > 0) {
    int da = db - 1;
    int64_t group = g.b[da];
    while (da > 0 && group * g.b[da - 1] <= target) {
      --da;
      group *= g.b[da];
    }
    if (group > cap) return false;
    rsft::FftPass ps{};
    ps.da = da;
    ps.db = db;
    ps.group = group;
    ps.inner = 1;
    for (int e = db; e < g.ndim; ++e) ps.inner *= g.b[e];
    ps.outer = 1;
    for (int e = 0; e < da; ++e) ps.outer *= g.b[e];
    ps.width = std::min<int64_t>(ps.inner, std::max<int64_t>(1, target / group));
    ps.outer_per_cta = 1;
    if (ps.width == ps.inner) ps.outer_per_cta = std::min<int64_t>(ps.outer, std::max<int64_t>(1, target / (group * ps.inner)));
    ps.ctas_per_loop = (ps.outer / ps.outer_per_cta) * (ps.inner / ps.width);
    ps.last = (db == g.ndim) ? 1 : 0;
    passes.insert(passes.begin(), ps);
    db = da;
  }
  return true;
}

// Device workspace of one execution lane (buckets, detections, votes, row lists) and its
// 16-byte count block (located count, error flag).
// Partial sums a chunked fold schedule leaves for fold_reduce (0 for direct schedules).
int64_t partial_elems(const rsft::FoldSchedule& fs, int loops) {
  if (fs.direct) return 0;
  return static_cast<int64_t>(std::min(loops, rsft::kMaxLoopGroup)) * fs.classes * fs.row_chunks * fs.col_chunks *
         fs.xcount;
}

// Frees one of the plan's own device allocations (NULL is a no-op).
void free_alloc(rsft_plan* p, const void* ptr) {
  if (!ptr) return;
  auto it = std::find(p->allocations.begin(), p->allocations.end(), const_cast<void*>(ptr));
  if (it == p->allocations.end()) return;
  cudaFree(*it);
  p->allocations.erase(it);
}

rsft_status alloc_workspace(rsft_plan* p, rsft::Workspace& ws, int64_t** d_count) {
  const rsft::HostPlan& h = p->host;
  const int L = h.loops;
  rsft_status st;
  const size_t lb = static_cast<size_t>(L) * h.total_b;
  if ((st = dev_alloc(p, &ws.folded, lb * sizeof(float2))) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &ws.spectrum, lb * sizeof(float2))) != RSFT_OK) return st;
  ws.partial = nullptr;
  p->partial_cap = std::max(p->partial_cap, partial_elems(p->fold, L));
  if (p->partial_cap > 0 &&
      (st = dev_alloc(p, &ws.partial, static_cast<size_t>(p->partial_cap) * sizeof(float2))) != RSFT_OK)
    return st;
  ws.words_b = (h.total_b + 31) / 32;
  // rounded up to 16 bytes: the vote kernel stages the bitmaps with one bulk copy
  if ((st = dev_alloc(p, &ws.det_bits, (static_cast<size_t>(L) * ws.words_b * 4 + 15) & ~static_cast<size_t>(15))) !=
      RSFT_OK)
    return st;
  if ((st = dev_alloc(p, &ws.det_count, static_cast<size_t>(L) * 4)) != RSFT_OK) return st;
  ws.gamma_used = nullptr;
  if (h.estimate_noise) {
    if ((st = dev_alloc(p, &ws.gamma_used, static_cast<size_t>(L) * 4)) != RSFT_OK) return st;
    std::vector<float> nan(L, std::numeric_limits<float>::quiet_NaN());
    cudaError_t ce = cudaMemcpy(ws.gamma_used, nan.data(), nan.size() * 4, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemcpy(gamma_used)");
  }
  ws.segments = rsft::stage2_segments(h.total_n);
  const size_t vote_bytes = static_cast<size_t>(ws.segments) * 16 * 1024;
  ws.vote_words = static_cast<int64_t>(vote_bytes / 4);
  if ((st = dev_alloc(p, &ws.votes, vote_bytes)) != RSFT_OK) return st;
  cudaError_t e = cudaMemset(ws.votes, 0, vote_bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(votes)");
  if ((st = dev_alloc(p, &ws.seg_count, static_cast<size_t>(ws.segments) * 4)) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &ws.seg_offset, static_cast<size_t>(ws.segments + 1) * 8)) != RSFT_OK) return st;
  if (p->rows_mode) {
    if ((st = dev_alloc(p, &ws.warp_count, static_cast<size_t>(p->rows.warps) * 4)) != RSFT_OK) return st;
    if ((st = dev_alloc(p, &ws.warp_offset, static_cast<size_t>(p->rows.warps + 1) * 8)) != RSFT_OK) return st;
    if (p->rows.small) {
      const size_t entries = static_cast<size_t>(p->rows.warps) * p->rows.rows_per_warp;
      if ((st = dev_alloc(p, &ws.row_list, entries * 16)) != RSFT_OK) return st;
      if ((st = dev_alloc(p, &ws.warp_rows, static_cast<size_t>(p->rows.warps) * 4)) != RSFT_OK) return st;
    }
  }
  if ((st = dev_alloc(p, d_count, 16)) != RSFT_OK) return st;
  ws.err_flag = reinterpret_cast<int*>(*d_count + 1);  // [1] of the count block
  e = cudaMemset(*d_count, 0, 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(flags)");
  return RSFT_OK;
}

// Fold tables in FP64, rounded once: per row the product of the row dimensions' weights
// a_{l,d}(s_d), w = c + jd, as one record per (row, class) (fold_record_f4: the pairs (d - c, c + d)
// of two loops per float4, then c of four loops per float4), and per column the product of the
// rest; loops grouped by `group` (one fold launch per group).
rsft_status build_fold_tables(rsft_plan* p, int group, rsft::DeviceTables& tabs) {
  const rsft::HostPlan& h = p->host;
  const int L = h.loops, D = h.ndim;
  rsft_status st;
  {
    const rsft::FoldSchedule& fs = p->fold;
    auto weight = [&](int l, int d, int64_t sd) {
      return h.wbar[d][(h.sigma_inv[l * D + d] * sd) & (h.n[d] - 1)] * h.w[d][sd];
    };
    // layout [class group][row chunk][stage][row slot][step][record]: a stage's records are
    // contiguous, and a row slot's records of consecutive steps adjacent
    const int64_t R = fs.rows_per_chunk, C = fs.cps;
    const int64_t spst = rsft::fold_stage_steps(fs), crow = fs.crow, rs = C * crow;
    const int64_t tunits = static_cast<int64_t>(fs.groups) * fs.row_chunks;
    const int full = std::min(group, L);
    const int64_t group_f4 = tunits * R * C * rsft::fold_record_f4(full);
    const int ngroups = (L + group - 1) / group;
    std::vector<float4> ft(static_cast<size_t>(group_f4) * ngroups, make_float4(0.f, 0.f, 0.f, 0.f));
    std::vector<float2> fc(static_cast<size_t>(L) * fs.col_chunks * fs.width);
    for (int l0 = 0; l0 < L; l0 += group) {
      const int lg = std::min(group, L - l0);
      const int rec = rsft::fold_record_f4(lg), npair = (lg + 1) / 2;
      const size_t tbase = static_cast<size_t>(l0 / group) * group_f4;
      for (int64_t e = 0; e < tunits * R * C; ++e) {
        const int64_t ci = e % C, r = (e / C) % R, tu = e / (C * R);
        const int64_t cls = (tu / fs.row_chunks) * C + ci, rc = tu % fs.row_chunks;
        int64_t sdig[rsft::kMaxDim] = {0, 0, 0, 0};
        int64_t rr = rc * R + r, cres = cls;
        for (int d = fs.d_in - 1; d >= 0; --d) {
          const int64_t md = rr % h.m[d], xd = cres % h.b[d];
          rr /= h.m[d];
          cres /= h.b[d];
          sdig[d] = xd + h.b[d] * md;
        }
        const int64_t stage = r / (spst * crow), step = (r / crow) % spst, ro = (r % crow) * C + ci;
        const int64_t at = tu * R * C + (stage * rs + ro) * spst + step;   // record index in the group
        float* out = reinterpret_cast<float*>(&ft[tbase + static_cast<size_t>(at) * rec]);
        for (int l = 0; l < lg; ++l) {
          cplx wv(1.0, 0.0);
          for (int d = 0; d < fs.d_in; ++d) wv *= weight(l0 + l, d, sdig[d]);
          out[2 * l] = static_cast<float>(wv.imag() - wv.real());      // pair float4 l / 2, half l % 2
          out[2 * l + 1] = static_cast<float>(wv.real() + wv.imag());
          out[4 * npair + l] = static_cast<float>(wv.real());           // c-value float4 l / 4, lane l % 4
        }
      }
      const size_t cbase = static_cast<size_t>(l0) * fs.col_chunks * fs.width;
      for (int cc = 0; cc < fs.col_chunks; ++cc)
        for (int l = 0; l < lg; ++l)
          for (int c = 0; c < fs.width; ++c) {
            int64_t col = static_cast<int64_t>(cc) * fs.width + c;
            cplx wv(1.0, 0.0);
            for (int d = D - 1; d >= fs.d_in; --d) {
              const int64_t sd = col % h.n[d];
              col /= h.n[d];
              wv *= weight(l0 + l, d, sd);
            }
            fc[cbase + (static_cast<size_t>(cc) * lg + l) * fs.width + c] = to_f2(wv);
          }
    }
    float4* f4 = nullptr;
    if ((st = upload(p, &f4, ft)) != RSFT_OK) return st;
    tabs.ftable = f4;
    tabs.ftable_group_f4 = group_f4;
    tabs.ftable_group = group;
    float2* f2p = nullptr;
    if ((st = upload(p, &f2p, fc)) != RSFT_OK) return st;
    tabs.fcolw = f2p;
  }
  return RSFT_OK;
}

// Everything that depends on the fold schedule p->fold: the epilogue's partial-sum slots
// per (class, residue), the residue digits, the tensor-core choice and the fold tables
// (segment-mode tables are rebuilt on their next use).
rsft_status apply_fold_schedule(rsft_plan* p) {
  const rsft::HostPlan& h = p->host;
  const rsft::Geometry& g = p->geom;
  const int L = h.loops, D = h.ndim;
  rsft_status st;
  // the previous schedule's tables (a re-tuned plan), and segment tables built from them
  if (p->seg_ready) {
    free_alloc(p, p->seg_tables.ftable);
    free_alloc(p, p->seg_tables.fcolw);
  }
  p->seg_ready = false;
  free_alloc(p, p->tables.ftable);
  free_alloc(p, p->tables.fcolw);
  free_alloc(p, p->tables.slots_by_x);
  free_alloc(p, p->tables.x_digits);
  p->tables.ftable = nullptr;
  p->tables.fcolw = nullptr;
  p->tables.slots_by_x = nullptr;
  p->tables.x_digits = nullptr;
  // fold epilogue tables: the partial sums left after the warp shuffle, grouped by the
  // inner residue of their columns, and the residue digits of each inner residue
  {
    rsft::FoldSchedule& fs = p->fold;
    std::vector<unsigned short> cols, digits;
    if (const char* why = rsft::fold_epilogue_tables(h.n, h.b, D, fs, cols, digits))
      return fail(RSFT_ERR_UNSUPPORTED, why);
    unsigned short* up = nullptr;
    if ((st = upload(p, &up, cols)) != RSFT_OK) return st;
    p->tables.slots_by_x = up;
    if ((st = upload(p, &up, digits)) != RSFT_OK) return st;
    p->tables.x_digits = up;
    p->h_slots = cols;
    p->h_xdig = digits;
    p->tables.h_slots = p->h_slots.data();
    p->tables.h_xdig = p->h_xdig.data();
    if (rsft::fold_smem_bytes(g, fs, std::min(L, p->loop_group)) > 227 * 1024)
      return fail(RSFT_ERR_UNSUPPORTED, "fold schedule needs more shared memory than a CTA has");
    // the tensor-core fold (schedules of whole 64-column rows) on request: RSFT_FOLD=tc
    const char* env = std::getenv("RSFT_FOLD");
    p->fold_tc = rsft::fold_tc_supported(g, fs) && env && std::string(env) == "tc";
    p->h_xres.assign(64, 0);
    for (int c = 0; c < 64 && c < fs.width; ++c)
      p->h_xres[c] = static_cast<unsigned char>(rsft::fold_residue(h.n, h.b, D, fs, c));
    p->tables.h_xres = p->h_xres.data();
  }
  if ((st = build_fold_tables(p, p->loop_group, p->tables)) != RSFT_OK) return st;
  return RSFT_OK;
}

rsft_status build_device(rsft_plan* p) {
  const rsft::HostPlan& h = p->host;
  rsft::Geometry& g = p->geom;
  g.ndim = h.ndim;
  g.loops = h.loops;
  g.total_n = h.total_n;
  g.total_b = h.total_b;
  for (int d = 0; d < rsft::kMaxDim; ++d) {
    g.n[d] = d < h.ndim ? h.n[d] : 1;
    g.b[d] = d < h.ndim ? h.b[d] : 1;
    g.m[d] = d < h.ndim ? h.m[d] : 1;
    g.log_n[d] = ilog2(g.n[d]);
    g.log_b[d] = ilog2(g.b[d]);
    g.log_m[d] = ilog2(g.m[d]);
  }
  for (int d = 0; d < rsft::kMaxDim; ++d) {
    g.n_shift[d] = 0;
    g.b_shift[d] = 0;
    for (int e = d + 1; e < h.ndim; ++e) {
      g.n_shift[d] += g.log_n[e];
      g.b_shift[d] += g.log_b[e];
    }
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  p->sms = sms;
  if (!rsft::choose_fold_schedule(g, sms, p->fold))
    return fail(RSFT_ERR_UNSUPPORTED, "no fold schedule for this bucket grid (inner B_d too large)");
  p->rows = rsft::VoteRowSchedule{};
  p->rows_mode = h.desc.vote_mode == RSFT_VOTES_ROWS && choose_vote_rows(g, p->rows) &&
                 static_cast<int64_t>(8) * ((p->rows.n_in + 3) / 4) * 4 <= 200 * 1024;
  if (!plan_fft_passes(g, p->passes))
    return fail(RSFT_ERR_UNSUPPORTED, "a bucket dimension is too large for the shared-memory FFT");
  {
    // one cluster launch for the bucket FFT where the grid allows it; RSFT_FFT=passes keeps the passes
    const char* env = std::getenv("RSFT_FFT");
    p->fft_cluster = rsft::fft_cluster_size(g) > 0 && !(env && std::string(env) == "passes");
  }

  const int L = h.loops, D = h.ndim;
  rsft_status st;
  // per-loop, per-dimension fold weights a_{l,d}(s) = w-bar_d(sigma^{-1} s mod N_d) w_d(s)
  for (int d = 0; d < D; ++d) {
    const int64_t n = h.n[d];
    std::vector<float2> tab(static_cast<size_t>(L) * n);
    for (int l = 0; l < L; ++l) {
      const int64_t si = h.sigma_inv[l * D + d];
      for (int64_t s = 0; s < n; ++s) tab[l * n + s] = to_f2(h.wbar[d][(si * s) & (n - 1)] * h.w[d][s]);
    }
    float2* dp = nullptr;
    if ((st = upload(p, &dp, tab)) != RSFT_OK) return st;
    p->tables.wtab[d] = dp;
    // grouped by residue class: [x][l][m] = a_{l,d}(x + B_d m), contiguous per class
    std::vector<float2> cls(static_cast<size_t>(L) * n);
    const int64_t bd = h.b[d], md = h.m[d];
    for (int64_t x = 0; x < bd; ++x)
      for (int l = 0; l < L; ++l)
        for (int64_t m = 0; m < md; ++m) cls[(x * L + l) * md + m] = tab[l * n + x + bd * m];
    if ((st = upload(p, &dp, cls)) != RSFT_OK) return st;
    p->tables.wcls[d] = dp;
    // twiddles e^{-j 2 pi k / B_d}
    std::vector<float2> tw(std::max<int64_t>(1, h.b[d] / 2));
    for (int64_t k = 0; k < h.b[d] / 2; ++k)
      tw[k] = to_f2(std::polar(1.0, -2.0 * 3.14159265358979323846 * static_cast<double>(k) / static_cast<double>(h.b[d])));
    if ((st = upload(p, &dp, tw)) != RSFT_OK) return st;
    p->tables.twiddle[d] = dp;
    // inverse pass-band gains; dimension 0 also carries 1 / prod_d sum w_d
    std::vector<float2> gi(h.m[d]);
    for (int64_t v = 0; v < h.m[d]; ++v) {
      cplx x = 1.0 / h.gain_pass[d][v];
      if (d == 0) x /= h.wsum;
      gi[v] = to_f2(x);
    }
    if ((st = upload(p, &dp, gi)) != RSFT_OK) return st;
    p->tables.ginv[d] = dp;
  }
  for (int d = D; d < rsft::kMaxDim; ++d) {
    p->tables.wtab[d] = nullptr;
    p->tables.wcls[d] = nullptr;
    p->tables.twiddle[d] = nullptr;
    p->tables.ginv[d] = nullptr;
  }
  std::vector<int> sg(L * D), si(L * D), sib(L * D);
  for (int l = 0; l < L; ++l)
    for (int d = 0; d < D; ++d) {
      sg[l * D + d] = static_cast<int>(h.sigma[l * D + d]);
      si[l * D + d] = static_cast<int>(h.sigma_inv[l * D + d]);
      sib[l * D + d] = static_cast<int>(h.sigma_inv[l * D + d] & (h.b[d] - 1));
    }
  int* ip = nullptr;
  if ((st = upload(p, &ip, sg)) != RSFT_OK) return st;
  p->tables.sigma = ip;
  if ((st = upload(p, &ip, si)) != RSFT_OK) return st;
  p->tables.sigma_inv = ip;
  if ((st = upload(p, &ip, sib)) != RSFT_OK) return st;
  p->tables.sigma_inv_b = ip;
  std::vector<float> gam(L);
  for (int l = 0; l < L; ++l) gam[l] = static_cast<float>(h.gamma[l]);
  float* fp = nullptr;
  if ((st = upload(p, &fp, gam)) != RSFT_OK) return st;
  p->tables.gamma = fp;
  p->h_sinvb = sib;
  p->tables.h_sinvb = p->h_sinvb.data();
  if ((st = apply_fold_schedule(p)) != RSFT_OK) return st;
  p->tables.rowmask = nullptr;
  p->tables.kb16 = nullptr;
  if (p->rows_mode && p->rows.small) {
    // candidate masks of the inner buckets of a row: bit i_in of mask[l][b] set iff the
    // inner candidates R(b, sigma_l^{-1}) (Def. 4, trailing dimensions) contain i_in
    const rsft::VoteRowSchedule& vs = p->rows;
    std::vector<uint64_t> masks(static_cast<size_t>(L) * vs.b_in, 0ull);
    for (int l = 0; l < L; ++l)
      for (int b = 0; b < vs.b_in; ++b)
        for (int u = 0; u < vs.m_in; ++u) {
          int64_t iin = 0, brem = b, urem = u, stride = 1;
          for (int d = D - 1; d >= vs.d_v; --d) {
            const int64_t bd = brem % h.b[d], ud = urem % h.m[d];
            brem /= h.b[d];
            urem /= h.m[d];
            const int64_t id = (h.sigma_inv[l * D + d] * (bd * h.m[d] + ud)) & (h.n[d] - 1);
            iin += id * stride;
            stride *= h.n[d];
          }
          masks[static_cast<size_t>(l) * vs.b_in + b] |= 1ull << iin;
        }
    if (vs.b_in <= 8) {
      // per loop, the union of the candidate masks of every detection pattern of a plane
      const int np = 1 << vs.b_in;
      std::vector<uint64_t> pat(static_cast<size_t>(L) * np, 0ull);
      for (int l = 0; l < L; ++l)
        for (int q = 1; q < np; ++q)
          for (int b = 0; b < vs.b_in; ++b)
            if ((q >> b) & 1) pat[static_cast<size_t>(l) * np + q] |= masks[static_cast<size_t>(l) * vs.b_in + b];
      masks.swap(pat);
    }
    uint64_t* mp = nullptr;
    if (masks.size() % 2) masks.push_back(0ull);  // whole 16-byte units for the bulk copy
    if ((st = upload(p, &mp, masks)) != RSFT_OK) return st;
    p->tables.rowmask = mp;
    // bucket-plane offsets of the row dimensions: ((sigma i mod N_d) >> log M_d) << b_shift_d (< B <= 65536)
    // per dimension [N_d][Lp]: the offsets of all loops of one index together, padded to eight
    const int Lp = (L + 7) & ~7;
    std::vector<uint16_t> kb;
    for (int d = 0; d < vs.d_v; ++d)
      for (int64_t i = 0; i < h.n[d]; ++i)
        for (int l = 0; l < Lp; ++l)
          kb.push_back(l < L ? static_cast<uint16_t>((((h.sigma[l * D + d] * i) & (h.n[d] - 1)) >> p->geom.log_m[d])
                                                     << p->geom.b_shift[d])
                             : static_cast<uint16_t>(0));
    while (kb.empty() || kb.size() % 8 != 0) kb.push_back(0u);  // whole 16-byte units for the bulk copy
    uint16_t* kp = nullptr;
    if ((st = upload(p, &kp, kb)) != RSFT_OK) return st;
    p->tables.kb16 = kp;
  }
  // workspace of lane 0
  p->ws.words_b = (h.total_b + 31) / 32;
  if (p->rows_mode && p->rows.small) {
    // one wave of resident blocks: each block stages its tables once
    int per_sm = 0, sms = 0;
    cudaError_t oe = rsft::vote_rows_small_residency(g, p->rows, p->ws.words_b, &per_sm);
    if (oe == cudaSuccess) oe = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (oe != cudaSuccess) return cuda_fail(oe, "vote kernel residency");
    const int64_t resident_warps = static_cast<int64_t>(std::max(per_sm, 8)) * sms;
    int64_t rpw = (p->rows.rows + resident_warps - 1) / resident_warps;
    rpw = std::max<int64_t>(32, (rpw + 31) / 32 * 32);
    p->rows.rows_per_warp = static_cast<int>(rpw);
    p->rows.warps = (p->rows.rows + rpw - 1) / rpw;
  }
  if ((st = alloc_workspace(p, p->ws, &p->d_count)) != RSFT_OK) return st;
  cudaError_t e;
  e = cudaMallocHost(reinterpret_cast<void**>(&p->h_count), 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "plan upload");
  return RSFT_OK;
}

cudaEvent_t take_event(rsft_plan* p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Sum the elapsed times of all pending timed executes (waits for them).
void drain_timing(rsft_plan* p) {
  for (auto& ev : p->pending) {
    bool ok = true;
    for (cudaEvent_t e : ev) ok = ok && e != nullptr;
    if (ok && cudaEventSynchronize(ev[5]) == cudaSuccess) {
      float ms = 0.f;
      for (int s = 0; s < 5; ++s)
        if (cudaEventElapsedTime(&ms, ev[s], ev[s + 1]) == cudaSuccess) p->stage_ms[s] += ms;
      if (cudaEventElapsedTime(&ms, ev[0], ev[5]) == cudaSuccess) p->stage_ms[5] += ms;
      p->timed_executes += 1;
    }
    cudaGetLastError();
    for (cudaEvent_t e : ev)
      if (e) p->event_pool.push_back(e);
  }
  p->pending.clear();
  for (auto& ft : p->frames_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(ft.end) == cudaSuccess && cudaEventElapsedTime(&ms, ft.start, ft.end) == cudaSuccess) {
      p->frames_fold_ms += ms;
      p->frames_folded += ft.frames;
      p->frames_fold_launches += 1.0;
    }
    cudaGetLastError();
    p->event_pool.push_back(ft.start);
    p->event_pool.push_back(ft.end);
  }
  p->frames_pending.clear();
}

// Kernels one execute with a located list and amplitudes launches (no full vote array): the
// fold (and its reduce for chunked schedules) per loop group, the FFT, the noise floor in
// estimate mode, the votes and second stage (small rows: count and emit; wide rows: count, scan
// and write; scatter mode: scatter, count, scan and write), the median.
int launches_per_execute(const rsft_plan* p) {
  const int groups = (p->geom.loops + p->loop_group - 1) / p->loop_group;
  return groups * (p->fold.direct ? 1 : 2) + (p->fft_cluster ? 1 : static_cast<int>(p->passes.size())) +
         (p->host.estimate_noise && !p->fft_cluster ? 1 : 0) +
         (p->rows_mode ? (p->rows.small ? 2 : 3) : 4) + 1;
}

void release(rsft_plan* p) {
  if (!p) return;
  if (p->has_device) {
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    p->pending.clear();
    for (auto& ft : p->frames_pending) {
      if (ft.start) cudaEventDestroy(ft.start);
      if (ft.end) cudaEventDestroy(ft.end);
    }
    p->frames_pending.clear();
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    for (rsft_lane& ln : p->lanes) {
      if (ln.stream) cudaStreamDestroy(ln.stream);
      if (ln.done) cudaEventDestroy(ln.done);
      if (ln.h_count) cudaFreeHost(ln.h_count);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    for (void* a : p->allocations) cudaFree(a);
    if (p->h_count) cudaFreeHost(p->h_count);
    cudaGetLastError();
  }
  delete p;
}

// One fold launch of loops [l0, l0 + lg): the tensor-core fold where the plan has one, else
// the SIMT fold (and its partial-sum reduction when the schedule chunks rows or columns).
// One fold launch of loops [l0, l0 + lg).  `clear`: the SIMT fold also zeroes the detection
// bitmaps and counts (the first launch of an execute); the tensor-core fold leaves that to a memset.
cudaError_t fold_group(rsft_plan* p, const rsft::DeviceTables& ft, bool tensor_cores, const void* cube, int l0,
                       int lg, rsft::Workspace& ws, cudaStream_t stream, bool clear = false) {
  const rsft::Geometry& g = p->geom;
  if (tensor_cores) {
    cudaError_t e = cudaSuccess;
    if (clear) {
      e = cudaMemsetAsync(ws.det_bits, 0, static_cast<size_t>(g.loops) * ws.words_b * 4, stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(ws.det_count, 0, static_cast<size_t>(g.loops) * 4, stream);
      if (e != cudaSuccess) return e;
    }
    return rsft::launch_fold_tc(g, p->fold, ft, static_cast<const float2*>(cube), l0, lg, ws.folded, ws.err_flag,
                                &p->fold_copy_mode, stream);
  }
  rsft::FoldClear fc;
  if (clear) {
    fc.a = ws.det_bits;
    fc.na = static_cast<int64_t>(g.loops) * ws.words_b;
    fc.b = ws.det_count;
    fc.nb = g.loops;
  }
  cudaError_t e = rsft::launch_fold(g, p->fold, ft, static_cast<const float2*>(cube), l0, lg, ws.folded, ws.partial,
                                    ws.err_flag, &p->fold_copy_mode, stream, fc);
  if (e == cudaSuccess && !p->fold.direct) e = rsft::launch_fold_reduce(g, p->fold, ft, l0, lg, ws.partial, ws.folded, stream);
  return e;
}

rsft_status run_lane(rsft_plan* p, rsft::Workspace& ws, bool& votes_dirty, bool timed, const void* d_cube,
                     cudaStream_t stream, uint64_t* d_located, uint8_t* d_located_votes, float2* d_amp,
                     uint8_t* d_votes_out, int64_t* d_count, const void* const* d_segments = nullptr) {
  const rsft::Geometry& g = p->geom;
  cudaError_t e;
  if (d_segments) {
    for (int l = 0; l < g.loops; ++l)
      if (!d_segments[l] || reinterpret_cast<uintptr_t>(d_segments[l]) % 16 != 0)
        return fail(RSFT_ERR_INVALID_ARG, "every segment must be non-NULL and 16-byte aligned");
  } else if (reinterpret_cast<uintptr_t>(d_cube) % 16 != 0) {
    return fail(RSFT_ERR_INVALID_ARG, "cube must be 16-byte aligned");
  }
  std::array<cudaEvent_t, 6> ev{};
  timed = timed && p->timing;
  if (timed)
    for (auto& x : ev) x = take_event(p);
  auto mark = [&](int i) {
    if (timed && ev[i]) cudaEventRecord(ev[i], stream);
  };
  if (votes_dirty) {
    e = cudaMemsetAsync(ws.votes, 0, static_cast<size_t>(ws.vote_words) * 4, stream);
    if (e != cudaSuccess) return cuda_fail(e, "clear votes");
  }
  mark(0);
  // segment mode: loop l folds its own segment (one loop per launch); otherwise every loop
  // group folds the same cube in one pass
  const int group = d_segments ? 1 : p->loop_group;
  const rsft::DeviceTables& ft = d_segments ? p->seg_tables : p->tables;
  for (int l0 = 0; l0 < g.loops; l0 += group) {
    const int lg = std::min(group, g.loops - l0);
    const void* cube = d_segments ? d_segments[l0] : d_cube;
    e = fold_group(p, ft, p->fold_tc && !d_segments, cube, l0, lg, ws, stream, l0 == 0);
    if (e != cudaSuccess) return cuda_fail(e, "permute_window_fold");
  }
  mark(1);
  const bool estimate = p->host.estimate_noise;
  if (p->fft_cluster) {
    // (estimate mode: each loop's noise floor is selected inside the cluster that holds its buckets)
    e = rsft::launch_fft_cluster(g, p->tables, ws.folded, ws.spectrum, ws.det_bits, ws.det_count, ws.words_b,
                                 !estimate, stream, 1, 0, p->fft_csize, p->fft_threads,
                                 estimate ? ws.gamma_used : nullptr, static_cast<float>(p->host.floor_factor));
    if (e != cudaSuccess) return cuda_fail(e, "bucket_fft/np_detect (cluster)");
  } else {
    for (size_t i = 0; i < p->passes.size(); ++i) {
      e = rsft::launch_fft_pass(g, p->passes[i], p->tables, i == 0 ? ws.folded : ws.spectrum, ws.spectrum,
                                ws.det_bits, ws.det_count, ws.words_b, !estimate, stream);
      if (e != cudaSuccess) return cuda_fail(e, "bucket_fft/np_detect");
    }
  }
  if (estimate && !p->fft_cluster) {
    // noise floor of each loop from its own bucket powers, then the detection against it
    e = rsft::launch_noise_floor(g, ws.spectrum, static_cast<float>(p->host.floor_factor), ws.gamma_used,
                                 ws.det_bits, ws.det_count, ws.words_b, stream);
    if (e != cudaSuccess) return cuda_fail(e, "np_detect (noise floor)");
  }
  mark(2);
  if (p->rows_mode) {
    mark(3);
    e = rsft::launch_vote_rows(g, p->rows, p->tables, ws.det_bits, ws.words_b, p->host.mu, ws.warp_count,
                               ws.warp_offset, d_located, d_located_votes, d_votes_out, p->host.desc.max_located,
                               d_count, ws.err_flag, ws.row_list, ws.warp_rows, stream);
    if (e != cudaSuccess) return cuda_fail(e, "vote_rows");
  } else {
    votes_dirty = true;
    e = rsft::launch_vote_scatter(g, p->tables, ws.det_bits, ws.words_b, ws.votes, stream);
    if (e != cudaSuccess) return cuda_fail(e, "vote_scatter");
    mark(3);
    e = rsft::launch_stage2(g, p->host.mu, ws, d_located, d_located_votes, d_votes_out, p->host.desc.max_located,
                            d_count, stream);
    if (e != cudaSuccess) return cuda_fail(e, "stage2_compact");
    votes_dirty = false;
  }
  mark(4);
  if (d_amp && p->host.desc.max_located > 0) {
    e = rsft::launch_median(g, p->tables, ws.spectrum, d_located, d_count, p->host.desc.max_located, d_amp, stream);
    if (e != cudaSuccess) return cuda_fail(e, "median_estimate");
  }
  mark(5);
  if (timed) p->pending.push_back(ev);
  return RSFT_OK;
}

rsft_status run(rsft_plan* p, const void* d_cube, cudaStream_t stream, uint64_t* d_located,
                uint8_t* d_located_votes, float2* d_amp, uint8_t* d_votes_out, int64_t* d_count) {
  return run_lane(p, p->ws, p->votes_dirty, true, d_cube, stream, d_located, d_located_votes, d_amp, d_votes_out,
                  d_count);
}

}  // namespace

namespace rsft {
void set_last_error(const char* msg) { g_last_error = msg; }

namespace {
std::mutex g_attr_mutex;
std::map<std::pair<int, const void*>, int> g_smem_limit;                  // (device, kernel) -> bytes set
std::map<std::tuple<int, const void*, int, int>, int> g_resident;         // (device, kernel, threads, bytes)
}  // namespace

cudaError_t ensure_smem_limit(const void* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  int& cur = g_smem_limit[{dev, func}];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t device_resident_ctas(const void* func, int threads, int bytes, int* ctas) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    auto it = g_resident.find({dev, func, threads, bytes});
    if (it != g_resident.end()) {
      *ctas = it->second;
      return cudaSuccess;
    }
  }
  if ((e = ensure_smem_limit(func, bytes)) != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, static_cast<size_t>(bytes));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  g_resident[{dev, func, threads, bytes}] = per_sm * sms;
  *ctas = per_sm * sms;
  return cudaSuccess;
}
}  // namespace rsft

extern "C" {

void rsft_desc_init(rsft_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->ndim = 0;
  for (int i = 0; i < 4; ++i) {
    d->n[i] = 1;
    d->b[i] = 1;
    d->flat_support[i] = 0;
  }
  d->loops = 8;
  d->window = RSFT_WIN_CHEB;
  d->atten_db = 60.0;
  d->flat = RSFT_FLAT_CHEB;
  d->p_fa = 1e-6;
  d->p_d = 0.9;
  d->k_max = 8;
  d->eta_p = 1.0;
  d->p_fa1_override = -1.0;
  d->mu_override = -1;
  d->noise_var = 1.0;
  d->seed = 0;
  d->sigma = nullptr;
  d->beta_mode = RSFT_BETA_EXACT;
  d->max_located = 65536;
  d->device = 0;
  d->vote_mode = RSFT_VOTES_ROWS;
  d->design_mode = RSFT_DESIGN_NORMAL;
}

rsft_status rsft_plan_create(const rsft_desc* desc, rsft_plan** plan) {
  if (!plan) return fail(RSFT_ERR_INVALID_ARG, "plan is NULL");
  *plan = nullptr;
  if (!desc) return fail(RSFT_ERR_INVALID_ARG, "desc is NULL");
  rsft_plan* p = new (std::nothrow) rsft_plan();
  if (!p) return fail(RSFT_ERR_OOM, "host allocation");
  std::string err;
  rsft_status st = rsft::build_host_plan(*desc, p->host, err);
  if (st != RSFT_OK) {
    delete p;
    return fail(st, err);
  }
  if (desc->device >= 0) {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || desc->device >= count) {
      cudaGetLastError();
      delete p;
      return fail(RSFT_ERR_CUDA, std::string("no CUDA device ") + std::to_string(desc->device) +
                                     (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : ""));
    }
    p->has_device = true;
    p->device = desc->device;
    DeviceGuard guard(p->device);
    if (!guard.ok) {
      p->has_device = false;
      delete p;
      return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
    }
    st = build_device(p);
    if (st != RSFT_OK) {
      std::string msg = g_last_error;
      release(p);
      return fail(st, msg);
    }
  }
  *plan = p;
  g_last_error.clear();
  return RSFT_OK;
}

void rsft_plan_destroy(rsft_plan* plan) { release(plan); }

}  // extern "C"

namespace {

// Extra lanes 0..n-1 of batched executes (workspace, count block, stream), and with
// `staging` their device cube and output buffers.
rsft_status ensure_lanes(rsft_plan* p, int n, bool staging) {
  rsft_status st;
  cudaError_t e;
  if (!p->fork && (e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_fail(e, "batch event");
  while (static_cast<int>(p->lanes.size()) < n) {
    rsft_lane ln;
    if ((st = alloc_workspace(p, ln.ws, &ln.d_count)) != RSFT_OK) return st;
    if ((e = cudaStreamCreateWithFlags(&ln.stream, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "lane stream");
    if ((e = cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming)) != cudaSuccess) {
      cudaStreamDestroy(ln.stream);
      return cuda_fail(e, "lane event");
    }
    if ((e = cudaMallocHost(reinterpret_cast<void**>(&ln.h_count), 16)) != cudaSuccess) {
      cudaStreamDestroy(ln.stream);
      cudaEventDestroy(ln.done);
      return cuda_fail(e, "lane count");
    }
    p->lanes.push_back(ln);
  }
  if (staging) {
    const int64_t cap = std::max<int64_t>(p->host.desc.max_located, 1);
    for (int i = 0; i < n; ++i) {
      rsft_lane& ln = p->lanes[i];
      if (ln.staging) continue;
      if ((st = dev_alloc(p, &ln.staging, static_cast<size_t>(p->host.total_n) * 8)) != RSFT_OK) return st;
      if ((st = dev_alloc(p, &ln.d_loc_stage, static_cast<size_t>(cap) * 8)) != RSFT_OK) return st;
      if ((st = dev_alloc(p, &ln.d_amp_stage, static_cast<size_t>(cap) * 8)) != RSFT_OK) return st;
    }
  }
  return RSFT_OK;
}

// Whether rsft_execute_frames runs frames together (one launch per stage over all frames): a
// direct SIMT fold schedule with every loop in one pass, the cluster FFT and the small-row votes.
bool frames_together(const rsft_plan* p) {
  return p->fold.direct && !p->fold_tc && p->loop_group >= p->host.loops && p->fft_cluster && p->rows_mode &&
         p->rows.small;
}

rsft_status ensure_frames(rsft_plan* p) {
  rsft_frame_work& fw = p->frames;
  if (fw.cap >= rsft::kMaxFrames) return RSFT_OK;
  const int F = rsft::kMaxFrames;
  const int L = p->host.loops;
  const size_t lb = static_cast<size_t>(L) * p->host.total_b;
  const int64_t words_b = p->ws.words_b;
  fw.frame_bits = (static_cast<int64_t>(L) * words_b + 3) & ~int64_t(3);
  rsft_status st;
  if ((st = dev_alloc(p, &fw.folded, F * lb * sizeof(float2))) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &fw.spectrum, F * lb * sizeof(float2))) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &fw.det_bits, static_cast<size_t>(F) * fw.frame_bits * 4)) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &fw.det_count, static_cast<size_t>(F) * L * 4)) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &fw.gamma_used, static_cast<size_t>(F) * L * 4)) != RSFT_OK) return st;
  const size_t warps = static_cast<size_t>(p->rows.warps);
  if ((st = dev_alloc(p, &fw.warp_count, F * warps * 4)) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &fw.warp_rows, F * warps * 4)) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &fw.row_list, F * warps * p->rows.rows_per_warp * 16)) != RSFT_OK) return st;
  fw.cap = F;
  return RSFT_OK;
}

// Frames [0, n) of one plan, kMaxFrames per launch of each stage: frame f reads d_cubes[f] and
// writes d_located + f * max_located, d_amp + f * max_located and d_counts[f].
rsft_status run_frames(rsft_plan* p, const void* const* d_cubes, int64_t n, cudaStream_t s, uint64_t* d_located,
                       float2* d_amp, int64_t* d_counts, bool timed) {
  const rsft::ChainLaunches unchained(false);  // frame groups of two plans share the GPU
  const rsft::Geometry& g = p->geom;
  const int L = g.loops;
  const int64_t cap = p->host.desc.max_located;
  rsft_frame_work& fw = p->frames;
  const int64_t words_b = p->ws.words_b;
  const bool estimate = p->host.estimate_noise;
  cudaError_t e = cudaSuccess;
  for (int64_t f0 = 0; f0 < n; f0 += rsft::kMaxFrames) {
    const int nf = static_cast<int>(std::min<int64_t>(rsft::kMaxFrames, n - f0));
    rsft::FoldClear fc;  // the fold zeroes the group's detection bitmaps and counts
    fc.a = fw.det_bits;
    fc.na = static_cast<int64_t>(nf) * fw.frame_bits;
    fc.b = fw.det_count;
    fc.nb = static_cast<int64_t>(nf) * L;
    const float2* cubes[rsft::kMaxFrames];
    for (int f = 0; f < nf; ++f) cubes[f] = static_cast<const float2*>(d_cubes[f0 + f]);
    rsft_plan::FramesTiming ft{nullptr, nullptr, nf};
    if (timed && p->timing) {
      ft.start = take_event(p);
      ft.end = take_event(p);
      if (ft.start) cudaEventRecord(ft.start, s);
    }
    e = rsft::launch_fold_frames(g, p->fold, p->tables, cubes, nf, static_cast<int64_t>(L) * g.total_b, 0, L,
                                 fw.folded, nullptr, p->ws.err_flag, &p->fold_copy_mode, s, fc);
    if (e != cudaSuccess) return cuda_fail(e, "permute_window_fold (frames)");
    if (ft.start && ft.end) {
      cudaEventRecord(ft.end, s);
      p->frames_pending.push_back(ft);
    }
    // many frames' CTAs fill the GPU, so the FFT's CTAs go narrower (256 threads) unless the plan
    // fixes a shape: 16-frame groups of the radar cube 44.0 -> 43.1 us a frame, the batched shapes
    // equal or faster; the arithmetic does not depend on the shape
    e = rsft::launch_fft_cluster(g, p->tables, fw.folded, fw.spectrum, fw.det_bits, fw.det_count, words_b, !estimate,
                                 s, nf, fw.frame_bits, p->fft_csize, p->fft_threads ? p->fft_threads : 256,
                                 estimate ? fw.gamma_used : nullptr, static_cast<float>(p->host.floor_factor));
    if (e != cudaSuccess) return cuda_fail(e, "bucket_fft/np_detect (frames)");
    if (estimate && !p->fft_cluster) {
      e = rsft::launch_noise_floor(g, fw.spectrum, static_cast<float>(p->host.floor_factor), fw.gamma_used,
                                   fw.det_bits, fw.det_count, words_b, s, nf, fw.frame_bits);
      if (e != cudaSuccess) return cuda_fail(e, "np_detect noise floor (frames)");
    }
    uint64_t* loc = d_located ? d_located + f0 * cap : nullptr;
    e = rsft::launch_vote_rows(g, p->rows, p->tables, fw.det_bits, words_b, p->host.mu, fw.warp_count, nullptr, loc,
                               nullptr, nullptr, cap, d_counts + f0, p->ws.err_flag, fw.row_list, fw.warp_rows, s, nf,
                               fw.frame_bits);
    if (e != cudaSuccess) return cuda_fail(e, "vote_rows (frames)");
    if (d_amp && cap > 0) {
      e = rsft::launch_median(g, p->tables, fw.spectrum, loc, d_counts + f0, cap, d_amp + f0 * cap, s, nf);
      if (e != cudaSuccess) return cuda_fail(e, "median_estimate (frames)");
    }
  }
  return RSFT_OK;
}

// Frames one after another on the plan's own workspace (plans whose stages cannot take several
// frames per launch).
rsft_status run_frames_in_turn(rsft_plan* p, const void* const* d_cubes, int64_t n, cudaStream_t s,
                               uint64_t* d_located, float2* d_amp, int64_t* d_counts) {
  const int64_t cap = p->host.desc.max_located;
  for (int64_t f = 0; f < n; ++f) {
    rsft_status st = run_lane(p, p->ws, p->votes_dirty, false, d_cubes[f], s, d_located ? d_located + f * cap : nullptr,
                              nullptr, d_amp ? d_amp + f * cap : nullptr, nullptr, d_counts + f);
    if (st != RSFT_OK) return st;
  }
  return RSFT_OK;
}

rsft_status check_frames_args(rsft_plan* plan, const void* const* d_cubes, int64_t n_frames, uint64_t* d_located,
                              int64_t* d_counts) {
  if (!plan || n_frames < 0 || (n_frames > 0 && (!d_cubes || !d_counts)))
    return fail(RSFT_ERR_INVALID_ARG, "NULL plan, cubes or counts, or negative frame count");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (plan->host.desc.max_located > 0 && n_frames > 0 && !d_located) return fail(RSFT_ERR_INVALID_ARG, "d_located is NULL");
  for (int64_t f = 0; f < n_frames; ++f)
    if (!d_cubes[f] || reinterpret_cast<uintptr_t>(d_cubes[f]) % 16 != 0)
      return fail(RSFT_ERR_INVALID_ARG, "every cube must be non-NULL and 16-byte aligned");
  return RSFT_OK;
}

}  // namespace

extern "C" {

rsft_status rsft_execute_frames(rsft_plan* plan, const void* const* d_cubes, int64_t n_frames, void* stream,
                                uint64_t* d_located, void* d_amp, int64_t* d_counts) {
  rsft_status st = check_frames_args(plan, d_cubes, n_frames, d_located, d_counts);
  if (st != RSFT_OK || n_frames == 0) return st;
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!frames_together(plan))
    return run_frames_in_turn(plan, d_cubes, n_frames, s, d_located, static_cast<float2*>(d_amp), d_counts);
  if ((st = ensure_frames(plan)) != RSFT_OK) return st;
  return run_frames(plan, d_cubes, n_frames, s, d_located, static_cast<float2*>(d_amp), d_counts, true);
}

rsft_status rsft_plan_frames_together(const rsft_plan* plan, int32_t* together) {
  if (!plan || !together) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or output");
  *together = plan->has_device && frames_together(plan) ? 1 : 0;
  return RSFT_OK;
}

rsft_status rsft_execute_batch(rsft_plan* plan, const void* const* d_cubes, int64_t n_frames, int32_t lanes,
                               void* stream, uint64_t* d_located, void* d_amp, int64_t* d_counts) {
  if (!plan || (n_frames > 0 && (!d_cubes || !d_counts)) || n_frames < 0)
    return fail(RSFT_ERR_INVALID_ARG, "NULL plan, cubes or counts, or negative frame count");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (lanes < 1 || lanes > 8) return fail(RSFT_ERR_INVALID_ARG, "lanes must be 1..8");
  const int64_t cap = plan->host.desc.max_located;
  if (cap > 0 && n_frames > 0 && !d_located) return fail(RSFT_ERR_INVALID_ARG, "d_located is NULL");
  for (int64_t f = 0; f < n_frames; ++f)
    if (!d_cubes[f] || reinterpret_cast<uintptr_t>(d_cubes[f]) % 16 != 0)
      return fail(RSFT_ERR_INVALID_ARG, "every cube must be non-NULL and 16-byte aligned");
  if (n_frames == 0) return RSFT_OK;
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  const int nl = static_cast<int>(std::min<int64_t>(lanes, n_frames));
  rsft_status st = ensure_lanes(plan, nl, false);
  if (st != RSFT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventRecord(plan->fork, s);
  for (int i = 0; e == cudaSuccess && i < nl; ++i) e = cudaStreamWaitEvent(plan->lanes[i].stream, plan->fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch fork");
  for (int64_t f = 0; f < n_frames; ++f) {
    rsft_lane& ln = plan->lanes[f % nl];
    st = run_lane(plan, ln.ws, ln.votes_dirty, false, d_cubes[f], ln.stream, d_located ? d_located + f * cap : nullptr,
                  nullptr, d_amp ? static_cast<float2*>(d_amp) + f * cap : nullptr, nullptr, d_counts + f);
    if (st != RSFT_OK) return st;
  }
  for (int i = 0; e == cudaSuccess && i < nl; ++i) {
    e = cudaEventRecord(plan->lanes[i].done, plan->lanes[i].stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, plan->lanes[i].done, 0);
  }
  return e == cudaSuccess ? RSFT_OK : cuda_fail(e, "batch join");
}

static rsft_status finish_count(rsft_plan* plan, cudaStream_t s, int64_t* n_located, const char* what);

rsft_status rsft_execute_segments_async(rsft_plan* plan, const void* const* d_segments, void* stream,
                                        uint64_t* d_located, uint8_t* d_located_votes, void* d_amp,
                                        uint8_t* d_votes_out, int64_t* d_n_located) {
  if (!plan || !d_segments || !d_n_located) return fail(RSFT_ERR_INVALID_ARG, "NULL plan, segments or count");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (plan->host.desc.max_located > 0 && !d_located) return fail(RSFT_ERR_INVALID_ARG, "d_located is NULL");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  if (!plan->seg_ready) {
    plan->seg_tables = plan->tables;
    rsft_status st = build_fold_tables(plan, 1, plan->seg_tables);
    if (st != RSFT_OK) return st;
    plan->seg_ready = true;
  }
  return run_lane(plan, plan->ws, plan->votes_dirty, true, nullptr, static_cast<cudaStream_t>(stream), d_located,
                  d_located_votes, static_cast<float2*>(d_amp), d_votes_out, d_n_located, d_segments);
}

rsft_status rsft_execute_segments(rsft_plan* plan, const void* const* d_segments, void* stream, uint64_t* d_located,
                                  uint8_t* d_located_votes, void* d_amp, uint8_t* d_votes_out, int64_t* n_located) {
  if (!plan || !n_located) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or n_located");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  rsft_status st = rsft_execute_segments_async(plan, d_segments, stream, d_located, d_located_votes, d_amp,
                                               d_votes_out, plan->d_count);
  if (st != RSFT_OK) return st;
  return finish_count(plan, static_cast<cudaStream_t>(stream), n_located, "rsft_execute_segments");
}

rsft_status rsft_execute_host_batch(rsft_plan* plan, const void* const* h_cubes, int64_t n_frames, void* stream,
                                    uint64_t* h_located, void* h_amp, int64_t* h_counts) {
  if (!plan || n_frames < 0 || (n_frames > 0 && (!h_cubes || !h_counts)))
    return fail(RSFT_ERR_INVALID_ARG, "NULL plan, cubes or counts, or negative frame count");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  const int64_t cap = plan->host.desc.max_located;
  if (cap > 0 && n_frames > 0 && !h_located) return fail(RSFT_ERR_INVALID_ARG, "h_located is NULL");
  for (int64_t f = 0; f < n_frames; ++f)
    if (!h_cubes[f]) return fail(RSFT_ERR_INVALID_ARG, "NULL host cube");
  if (n_frames == 0) return RSFT_OK;
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  rsft_status st = ensure_lanes(plan, 2, true);
  if (st != RSFT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventRecord(plan->fork, s);
  for (int i = 0; e == cudaSuccess && i < 2; ++i) e = cudaStreamWaitEvent(plan->lanes[i].stream, plan->fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch fork");
  const size_t cube_bytes = static_cast<size_t>(plan->host.total_n) * 8;
  // frame f on lane f % 2: copy in, RSFT, count out; its lists follow once the count is known
  auto enqueue = [&](int64_t f) -> rsft_status {
    rsft_lane& ln = plan->lanes[f % 2];
    cudaError_t ce = cudaMemcpyAsync(ln.staging, h_cubes[f], cube_bytes, cudaMemcpyHostToDevice, ln.stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "copy cube to device");
    rsft_status rs = run_lane(plan, ln.ws, ln.votes_dirty, false, ln.staging, ln.stream, ln.d_loc_stage, nullptr,
                              h_amp ? ln.d_amp_stage : nullptr, nullptr, ln.d_count);
    if (rs != RSFT_OK) return rs;
    ce = cudaMemcpyAsync(ln.h_count, ln.d_count, 16, cudaMemcpyDeviceToHost, ln.stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(ln.done, ln.stream);
    return ce == cudaSuccess ? RSFT_OK : cuda_fail(ce, "copy count to host");
  };
  if ((st = enqueue(0)) != RSFT_OK) return st;
  rsft_status result = RSFT_OK;
  for (int64_t f = 0; f < n_frames; ++f) {
    if (f + 1 < n_frames && (st = enqueue(f + 1)) != RSFT_OK) return st;
    rsft_lane& ln = plan->lanes[f % 2];
    if ((e = cudaEventSynchronize(ln.done)) != cudaSuccess) return cuda_fail(e, "rsft_execute_host_batch");
    if (reinterpret_cast<const int*>(ln.h_count + 1)[0] != 0) {
      cudaMemsetAsync(ln.ws.err_flag, 0, sizeof(int), ln.stream);
      result = fail(RSFT_ERR_TIMEOUT, "a device wait gave up (error flag set)");
    }
    const int64_t c = ln.h_count[0];
    h_counts[f] = c;
    const int64_t k = std::min(c, cap);
    if (k > 0) {
      e = cudaMemcpyAsync(h_located + f * cap, ln.d_loc_stage, static_cast<size_t>(k) * 8, cudaMemcpyDeviceToHost,
                          ln.stream);
      if (e == cudaSuccess && h_amp)
        e = cudaMemcpyAsync(static_cast<float2*>(h_amp) + f * cap, ln.d_amp_stage, static_cast<size_t>(k) * 8,
                            cudaMemcpyDeviceToHost, ln.stream);
      if (e != cudaSuccess) return cuda_fail(e, "copy results to host");
    }
    if (c > cap && result == RSFT_OK) result = fail(RSFT_ERR_CAPACITY, "a located list was truncated to max_located");
  }
  for (int i = 0; i < 2; ++i)
    if ((e = cudaStreamSynchronize(plan->lanes[i].stream)) != cudaSuccess) return cuda_fail(e, "rsft_execute_host_batch");
  return result;
}

rsft_status rsft_execute_async(rsft_plan* plan, const void* d_cube, void* stream, uint64_t* d_located,
                               uint8_t* d_located_votes, void* d_amp, uint8_t* d_votes_out,
                               int64_t* d_n_located) {
  if (!plan || !d_cube || !d_n_located) return fail(RSFT_ERR_INVALID_ARG, "NULL plan, cube or count");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (plan->host.desc.max_located > 0 && !d_located) return fail(RSFT_ERR_INVALID_ARG, "d_located is NULL");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  return run(plan, d_cube, static_cast<cudaStream_t>(stream), d_located, d_located_votes,
             static_cast<float2*>(d_amp), d_votes_out, d_n_located);
}

// Reads the located count (and error flag) of the plan's own lane after an execute queued
// on `s`: TIMEOUT when a device wait gave up, CAPACITY when the list was truncated.
static rsft_status finish_count(rsft_plan* plan, cudaStream_t s, int64_t* n_located, const char* what) {
  DeviceGuard guard(plan->device);
  cudaError_t e = cudaMemcpyAsync(plan->h_count, plan->d_count, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, what);
  *n_located = *plan->h_count;
  if (reinterpret_cast<const int*>(plan->h_count + 1)[0] != 0) {
    cudaMemsetAsync(plan->ws.err_flag, 0, sizeof(int), s);
    return fail(RSFT_ERR_TIMEOUT, "a bounded device wait gave up (results invalid)");
  }
  if (*n_located > plan->host.desc.max_located)
    return fail(RSFT_ERR_CAPACITY, "located list truncated to max_located");
  return RSFT_OK;
}

rsft_status rsft_execute(rsft_plan* plan, const void* d_cube, void* stream, uint64_t* d_located,
                         uint8_t* d_located_votes, void* d_amp, uint8_t* d_votes_out, int64_t* n_located) {
  if (!plan || !n_located) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or n_located");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  rsft_status st = rsft_execute_async(plan, d_cube, stream, d_located, d_located_votes, d_amp, d_votes_out,
                                      plan->d_count);
  if (st != RSFT_OK) return st;
  return finish_count(plan, static_cast<cudaStream_t>(stream), n_located, "rsft_execute");
}

rsft_status rsft_execute_host(rsft_plan* plan, const void* h_cube, void* stream, uint64_t* h_located,
                              void* h_amp, int64_t* n_located) {
  if (!plan || !h_cube || !n_located) return fail(RSFT_ERR_INVALID_ARG, "NULL plan, cube or count");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  const int64_t cap = plan->host.desc.max_located;
  if (cap > 0 && !h_located) return fail(RSFT_ERR_INVALID_ARG, "h_located is NULL");
  DeviceGuard guard(plan->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rsft_status st;
  const size_t cube_bytes = static_cast<size_t>(plan->host.total_n) * 8;
  if (!plan->staging) {
    if ((st = dev_alloc(plan, &plan->staging, cube_bytes)) != RSFT_OK) return st;
    if ((st = dev_alloc(plan, &plan->d_loc_stage, static_cast<size_t>(std::max<int64_t>(cap, 1)) * 8)) != RSFT_OK)
      return st;
    if ((st = dev_alloc(plan, &plan->d_amp_stage, static_cast<size_t>(std::max<int64_t>(cap, 1)) * 8)) != RSFT_OK)
      return st;
  }
  cudaError_t e = cudaMemcpyAsync(plan->staging, h_cube, cube_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy cube to device");
  st = run(plan, plan->staging, s, plan->d_loc_stage, nullptr, h_amp ? plan->d_amp_stage : nullptr, nullptr,
           plan->d_count);
  if (st != RSFT_OK) return st;
  e = cudaMemcpyAsync(plan->h_count, plan->d_count, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "rsft_execute_host");
  if (reinterpret_cast<const int*>(plan->h_count + 1)[0] != 0) {
    cudaMemsetAsync(plan->ws.err_flag, 0, sizeof(int), s);
    return fail(RSFT_ERR_TIMEOUT, "a bounded device wait gave up (results invalid)");
  }
  const int64_t cnt = *plan->h_count;
  const int64_t ncopy = std::min(cnt, cap);
  if (ncopy > 0) {
    e = cudaMemcpyAsync(h_located, plan->d_loc_stage, static_cast<size_t>(ncopy) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_amp)
      e = cudaMemcpyAsync(h_amp, plan->d_amp_stage, static_cast<size_t>(ncopy) * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "copy located to host");
  }
  *n_located = cnt;
  if (cnt > cap) return fail(RSFT_ERR_CAPACITY, "located list truncated to max_located");
  return RSFT_OK;
}

rsft_status rsft_plan_get(const rsft_plan* plan, int32_t what, void* out, size_t bytes) {
  if (!plan || !out) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or out");
  const rsft::HostPlan& h = plan->host;
  const int L = h.loops, D = h.ndim;
  auto need = [&](size_t n) { return bytes >= n; };
  switch (what) {
    case RSFT_GET_SIGMA:
    case RSFT_GET_SIGMA_INV: {
      const size_t n = static_cast<size_t>(L) * D * 8;
      if (!need(n)) break;
      std::memcpy(out, (what == RSFT_GET_SIGMA ? h.sigma : h.sigma_inv).data(), n);
      return RSFT_OK;
    }
    case RSFT_GET_GAMMA:
    case RSFT_GET_BETA: {
      const size_t n = static_cast<size_t>(L) * 8;
      if (!need(n)) break;
      std::memcpy(out, (what == RSFT_GET_GAMMA ? h.gamma : h.beta).data(), n);
      return RSFT_OK;
    }
    case RSFT_GET_MU:
      if (!need(4)) break;
      *static_cast<int32_t*>(out) = h.mu;
      return RSFT_OK;
    case RSFT_GET_PFA1:
    case RSFT_GET_ETA_M:
    case RSFT_GET_PD_BAR:
      if (!need(8)) break;
      *static_cast<double*>(out) = what == RSFT_GET_PFA1 ? h.pfa1 : (what == RSFT_GET_ETA_M ? h.eta_m : h.pd_bar);
      return RSFT_OK;
    case RSFT_GET_WINDOW: {
      size_t total = 0;
      for (int d = 0; d < D; ++d) total += h.w[d].size();
      if (!need(total * 8)) break;
      double* o = static_cast<double*>(out);
      for (int d = 0; d < D; ++d) o = std::copy(h.w[d].begin(), h.w[d].end(), o);
      return RSFT_OK;
    }
    case RSFT_GET_FLAT: {
      size_t total = 0;
      for (int d = 0; d < D; ++d) total += h.wbar[d].size();
      if (!need(total * 16)) break;
      double* o = static_cast<double*>(out);
      for (int d = 0; d < D; ++d)
        for (const cplx& v : h.wbar[d]) {
          *o++ = v.real();
          *o++ = v.imag();
        }
      return RSFT_OK;
    }
    case RSFT_GET_WARNINGS:
      if (!need(4)) break;
      *static_cast<int32_t*>(out) = h.warnings;
      return RSFT_OK;
    case RSFT_GET_SNR_DB: {
      if (!need(8)) break;
      rsft_plan* mp = const_cast<rsft_plan*>(plan);
      if (!mp->snr_cached) {
        mp->snr_db = rsft::design_snr_db(h);
        mp->snr_cached = true;
      }
      *static_cast<double*>(out) = mp->snr_db;
      return RSFT_OK;
    }
    case RSFT_GET_WORKSPACE_BYTES: {
      if (!need(8)) break;
      int64_t tot = 0;
      if (plan->has_device) {
        const rsft::Workspace& ws = plan->ws;
        tot += 2 * static_cast<int64_t>(L) * h.total_b * 8 + static_cast<int64_t>(L) * ws.words_b * 4 +
               ws.vote_words * 4 + ws.segments * 12;
        if (!plan->fold.direct)
          tot += static_cast<int64_t>(std::min(L, rsft::kMaxLoopGroup)) * plan->fold.classes *
                 plan->fold.row_chunks * plan->fold.col_chunks * plan->fold.xcount * 8;
      }
      *static_cast<int64_t*>(out) = tot;
      return RSFT_OK;
    }
    case RSFT_GET_STAGE_MS: {
      if (!need(64)) break;
      rsft_plan* mp = const_cast<rsft_plan*>(plan);
      if (mp->has_device) {
        DeviceGuard guard(mp->device);
        drain_timing(mp);
      }
      double* o = static_cast<double*>(out);
      for (int s = 0; s < 6; ++s) o[s] = mp->stage_ms[s];
      o[6] = static_cast<double>(mp->timed_executes);
      o[7] = mp->has_device ? static_cast<double>(launches_per_execute(mp)) : 0.0;
      return RSFT_OK;
    }
    case RSFT_GET_GAMMA_LAST: {
      const size_t n = static_cast<size_t>(L) * 8;
      if (!need(n)) break;
      double* o = static_cast<double*>(out);
      if (!h.estimate_noise || !plan->has_device) {
        std::copy(h.gamma.begin(), h.gamma.end(), o);
        return RSFT_OK;
      }
      DeviceGuard guard(plan->device);
      std::vector<float> g(L);
      cudaError_t e = cudaDeviceSynchronize();
      if (e == cudaSuccess) e = cudaMemcpy(g.data(), plan->ws.gamma_used, static_cast<size_t>(L) * 4, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "rsft_plan_get(GAMMA_LAST)");
      for (int l = 0; l < L; ++l) o[l] = static_cast<double>(g[l]);
      return RSFT_OK;
    }
    case RSFT_GET_FFT_SHAPE: {
      if (!need(8)) break;
      int32_t* o = static_cast<int32_t*>(out);
      const bool on = plan->has_device && plan->fft_cluster;
      o[0] = on ? (plan->fft_csize > 0 ? plan->fft_csize : rsft::fft_cluster_size(plan->geom)) : 0;
      const int64_t E = on && o[0] > 0 ? plan->geom.total_b / o[0] : 0;
      o[1] = on ? (plan->fft_threads > 0 ? plan->fft_threads : (E >= 2048 ? 512 : 256)) : 0;
      return RSFT_OK;
    }
    case RSFT_GET_FRAMES_FOLD: {
      if (!need(24)) break;
      rsft_plan* mp = const_cast<rsft_plan*>(plan);
      if (mp->has_device) {
        DeviceGuard guard(mp->device);
        drain_timing(mp);
      }
      double* o = static_cast<double*>(out);
      o[0] = mp->frames_fold_ms;
      o[1] = mp->frames_folded;
      o[2] = mp->frames_fold_launches;
      return RSFT_OK;
    }
    case RSFT_GET_FOLD_COPY:
      if (!need(4)) break;
      *static_cast<int32_t*>(out) = plan->fold_copy_mode;
      return RSFT_OK;
    case RSFT_GET_FOLD_BYTES: {
      if (!need(8)) break;
      const int groups = (L + plan->loop_group - 1) / plan->loop_group;
      *static_cast<int64_t*>(out) = groups * h.total_n * 8 + static_cast<int64_t>(L) * h.total_b * 8;
      return RSFT_OK;
    }
    default:
      return fail(RSFT_ERR_INVALID_ARG, "unknown rsft_plan_get item");
  }
  return fail(RSFT_ERR_INVALID_ARG, "output buffer too small");
}

rsft_status rsft_plan_timing(rsft_plan* plan, int32_t enable) {
  if (!plan) return fail(RSFT_ERR_INVALID_ARG, "NULL plan");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan");
  DeviceGuard guard(plan->device);
  drain_timing(plan);
  for (double& v : plan->stage_ms) v = 0.0;
  plan->timed_executes = 0;
  plan->timing = enable != 0;
  return RSFT_OK;
}

rsft_status rsft_copy_buckets(rsft_plan* plan, int32_t which, void* d_out, void* stream) {
  if (!plan || !d_out) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or output");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan");
  if (which != RSFT_BUCKETS_FOLDED && which != RSFT_BUCKETS_SPECTRUM) return fail(RSFT_ERR_INVALID_ARG, "which");
  DeviceGuard guard(plan->device);
  const size_t n = static_cast<size_t>(plan->host.loops) * plan->host.total_b * 8;
  cudaError_t e = cudaMemcpyAsync(d_out, which == RSFT_BUCKETS_FOLDED ? plan->ws.folded : plan->ws.spectrum, n,
                                  cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rsft_copy_buckets");
  return RSFT_OK;
}

rsft_status rsft_copy_detections(rsft_plan* plan, void* d_out, void* stream) {
  if (!plan || !d_out) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or output");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan");
  DeviceGuard guard(plan->device);
  const size_t n = static_cast<size_t>(plan->host.loops) * plan->ws.words_b * 4;
  cudaError_t e = cudaMemcpyAsync(d_out, plan->ws.det_bits, n, cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "rsft_copy_detections");
  return RSFT_OK;
}

}  // extern "C"

namespace {

// Refinement geometry and scratch for K tones (kept and grown by the plan).
rsft_status ensure_refine(rsft_plan* p, int64_t k) {
  rsft::RefineGeom& rg = p->refine_geom;
  const rsft::HostPlan& h = p->host;
  rg.ndim = h.ndim;
  rg.loops = h.loops;
  rg.total_b = h.total_b;
  rg.sumb = 0;
  for (int d = 0; d < rsft::kMaxDim; ++d) {
    rg.n[d] = p->geom.n[d];
    rg.b[d] = p->geom.b[d];
    rg.m[d] = p->geom.m[d];
    rg.b_shift[d] = p->geom.b_shift[d];
    rg.boff[d] = rg.sumb;
    if (d < h.ndim) rg.sumb += static_cast<int>(h.b[d]);
  }
  rsft::RefineWork& w = p->refine;
  if (w.k_cap >= k && w.gres) return RSFT_OK;
  if (w.gres) {
    // more tones than before: the smaller per-tone buffers may still be read by queued work
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "rsft_refine (growing the tone buffers)");
    for (const void* q : {static_cast<const void*>(w.gres), static_cast<const void*>(w.gder),
                          static_cast<const void*>(w.contr), static_cast<const void*>(w.lm_gh),
                          static_cast<const void*>(w.lm_freq), static_cast<const void*>(w.lm_amp)})
      free_alloc(p, q);
  }
  const int64_t kk = std::max<int64_t>(k, 16);
  rsft_status st;
  const size_t resp = static_cast<size_t>(h.loops) * kk * rg.sumb * sizeof(float2);
  if ((st = dev_alloc(p, &w.gres, resp)) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &w.gder, resp)) != RSFT_OK) return st;
  if (!w.resid) {
    if ((st = dev_alloc(p, &w.resid, static_cast<size_t>(h.loops) * h.total_b * sizeof(float2))) != RSFT_OK)
      return st;
    w.parts = 152 * 4;
    if ((st = dev_alloc(p, &w.partial, static_cast<size_t>(w.parts) * sizeof(double))) != RSFT_OK) return st;
  }
  const int vals = 3 + 5 * rsft::kMaxDim + rsft::kMaxDim * (rsft::kMaxDim - 1);
  if ((st = dev_alloc(p, &w.contr, static_cast<size_t>(h.loops) * kk * vals * sizeof(float))) != RSFT_OK)
    return st;
  if ((st = dev_alloc(p, &w.lm_gh, static_cast<size_t>(2) * kk * rsft::kLmTone * sizeof(double))) != RSFT_OK)
    return st;
  if ((st = dev_alloc(p, &w.lm_freq, static_cast<size_t>(kk) * rsft::kMaxDim * sizeof(float))) != RSFT_OK) return st;
  if ((st = dev_alloc(p, &w.lm_amp, static_cast<size_t>(kk) * sizeof(float2))) != RSFT_OK) return st;
  if (!w.lm_state && (st = dev_alloc(p, &w.lm_state, 8 * sizeof(double))) != RSFT_OK) return st;
  w.k_cap = kk;
  return RSFT_OK;
}

// The folded buckets F_l of the cube in the plan's workspace (the RSFT's own fold, all loops).
rsft_status fold_cube(rsft_plan* p, const void* d_cube, cudaStream_t stream) {
  if (reinterpret_cast<uintptr_t>(d_cube) % 16 != 0) return fail(RSFT_ERR_INVALID_ARG, "cube must be 16-byte aligned");
  const rsft::Geometry& g = p->geom;
  rsft::Workspace& ws = p->ws;
  for (int l0 = 0; l0 < g.loops; l0 += p->loop_group) {
    const int lg = std::min(p->loop_group, g.loops - l0);
    cudaError_t e = fold_group(p, p->tables, p->fold_tc, d_cube, l0, lg, ws, stream);
    if (e != cudaSuccess) return cuda_fail(e, "permute_window_fold");
  }
  return RSFT_OK;
}

}  // namespace

extern "C" {

rsft_status rsft_refine_prepare(rsft_plan* plan, const void* d_cube, void* stream) {
  if (!plan || !d_cube) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or cube");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  return fold_cube(plan, d_cube, static_cast<cudaStream_t>(stream));
}

rsft_status rsft_refine_eval(rsft_plan* plan, int64_t k, const float* d_freq, const void* d_amp, double* d_loss,
                             float* d_grad_freq, void* d_grad_amp, float* d_hdiag, void* stream) {
  if (!plan || k < 1 || !d_freq || !d_amp) return fail(RSFT_ERR_INVALID_ARG, "NULL plan, tones, or k < 1");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (k > (1 << 20)) return fail(RSFT_ERR_UNSUPPORTED, "more than 2^20 tones");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  rsft_status st = ensure_refine(plan, k);
  if (st != RSFT_OK) return st;
  cudaError_t e = rsft::launch_refine_eval(plan->refine_geom, plan->tables, plan->refine, plan->ws.folded,
                                           static_cast<int>(k), d_freq, static_cast<const float2*>(d_amp), d_loss,
                                           d_grad_freq, static_cast<float2*>(d_grad_amp), d_hdiag, nullptr,
                                           static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RSFT_OK : cuda_fail(e, "rsft_refine_eval");
}

rsft_status rsft_refine(rsft_plan* plan, const void* d_cube, int64_t k, float* d_freq, void* d_amp,
                        int32_t steps, float lr, void* stream) {
  if (!plan || !d_cube || k < 1 || !d_freq || !d_amp || steps < 0 || !(lr > 0.f))
    return fail(RSFT_ERR_INVALID_ARG, "NULL plan, cube or tones, k < 1, steps < 0 or lr <= 0");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (k > (1 << 20)) return fail(RSFT_ERR_UNSUPPORTED, "more than 2^20 tones");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rsft_status st = ensure_refine(plan, k);
  if (st == RSFT_OK) st = fold_cube(plan, d_cube, s);
  if (st != RSFT_OK) return st;
  // steps + 1 evaluations: the starting point, then one trial per step; the tones end at the
  // accepted point of lowest loss
  for (int it = 0; steps > 0 && it <= steps; ++it) {
    cudaError_t e = rsft::launch_refine_step(plan->refine_geom, plan->tables, plan->refine, plan->ws.folded,
                                             static_cast<int>(k), d_freq, static_cast<float2*>(d_amp), it, lr,
                                             it == steps, s);
    if (e != cudaSuccess) return cuda_fail(e, "rsft_refine");
  }
  return RSFT_OK;
}

rsft_status rsft_plan_set_loops_per_pass(rsft_plan* plan, int32_t loops_per_pass) {
  if (!plan) return fail(RSFT_ERR_INVALID_ARG, "NULL plan");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (loops_per_pass < 1 || loops_per_pass > rsft::kMaxLoopGroup)
    return fail(RSFT_ERR_INVALID_ARG, "loops per pass must be 1..16");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  cudaError_t e = cudaDeviceSynchronize();  // the old tables may still be read by queued work
  if (e != cudaSuccess) return cuda_fail(e, "rsft_plan_set_loops_per_pass");
  const int previous = plan->loop_group;
  plan->loop_group = loops_per_pass;
  const rsft_status st = apply_fold_schedule(plan);
  if (st != RSFT_OK) {
    plan->loop_group = previous;
    apply_fold_schedule(plan);
  }
  return st;
}

rsft_status rsft_plan_set_fft_shape(rsft_plan* plan, int32_t ctas_per_loop, int32_t threads) {
  if (!plan) return fail(RSFT_ERR_INVALID_ARG, "NULL plan");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan");
  if (ctas_per_loop == 0 && threads == 0) {
    plan->fft_csize = 0;
    plan->fft_threads = 0;
    return RSFT_OK;
  }
  if (!plan->fft_cluster) return fail(RSFT_ERR_UNSUPPORTED, "this plan's bucket FFT runs as shared-memory passes");
  if (!rsft::fft_cluster_valid(plan->geom, ctas_per_loop))
    return fail(RSFT_ERR_UNSUPPORTED, "CTAs per loop must be 1, 2, 4 or 8 and fit the bucket grid");
  if (threads != 256 && threads != 512) return fail(RSFT_ERR_INVALID_ARG, "threads must be 256 or 512");
  plan->fft_csize = ctas_per_loop;
  plan->fft_threads = threads;
  return RSFT_OK;
}

rsft_status rsft_plan_autotune(rsft_plan* plan, const void* d_cube, void* stream, int32_t candidates, int32_t reps,
                               double* us_out, int32_t* chosen) {
  if (!plan || !d_cube) return fail(RSFT_ERR_INVALID_ARG, "NULL plan or cube");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (candidates < 1 || candidates > 16 || reps < 1 || reps > 1000)
    return fail(RSFT_ERR_INVALID_ARG, "candidates must be 1..16 and reps 1..1000");
  if (reinterpret_cast<uintptr_t>(d_cube) % 16 != 0) return fail(RSFT_ERR_INVALID_ARG, "cube must be 16-byte aligned");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  std::vector<std::pair<double, rsft::FoldSchedule>> all;
  rsft::FoldSchedule model{};
  if (!rsft::choose_fold_schedule(plan->geom, plan->sms, model, &all, plan->loop_group))
    return fail(RSFT_ERR_UNSUPPORTED, "no fold schedule");
  std::stable_sort(all.begin(), all.end(),
                   [](const std::pair<double, rsft::FoldSchedule>& a, const std::pair<double, rsft::FoldSchedule>& b) {
                     return a.first < b.first;
                   });
  auto same = [](const rsft::FoldSchedule& a, const rsft::FoldSchedule& b) {
    return a.d_in == b.d_in && a.width == b.width && a.cps == b.cps && a.crow == b.crow && a.col_chunks == b.col_chunks;
  };
  std::vector<rsft::FoldSchedule> cands;
  for (const auto& c : all) {
    if (static_cast<int>(cands.size()) >= candidates) break;
    // chunked schedules need partial-sum buffers no larger than the workspaces already have
    if (partial_elems(c.second, plan->host.loops) > plan->partial_cap) continue;
    bool dup = false;
    for (const auto& k : cands) dup = dup || same(k, c.second);
    if (!dup) cands.push_back(c.second);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "autotune events");
  }
  const rsft::FoldSchedule original = plan->fold;
  double best_us = 1e300;
  int best = -1;
  rsft_status st = RSFT_OK;
  for (size_t i = 0; i < cands.size() && st == RSFT_OK; ++i) {
    plan->fold = cands[i];
    if (apply_fold_schedule(plan) != RSFT_OK) continue;  // e.g. more shared memory than a CTA has
    for (int w = 0; w < 2 && st == RSFT_OK; ++w) st = fold_cube(plan, d_cube, s);
    if (st != RSFT_OK) break;
    e = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == RSFT_OK; ++r) st = fold_cube(plan, d_cube, s);
    if (st != RSFT_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "autotune timing");
      break;
    }
    const double us = 1e3 * static_cast<double>(ms) / reps;
    if (us < best_us) {
      best_us = us;
      best = static_cast<int>(i);
    }
  }
  plan->fold = best >= 0 ? cands[best] : original;
  const rsft_status st2 = apply_fold_schedule(plan);
  // the bucket FFT's shape: CTAs per loop (buckets per CTA) and threads per CTA, timed on the
  // buckets of the cube under the chosen fold schedule
  if (st == RSFT_OK && st2 == RSFT_OK && best >= 0 && plan->fft_cluster) {
    st = fold_cube(plan, d_cube, s);
    const rsft::Geometry& g = plan->geom;
    double fft_best = 1e300;
    int bc = 0, bt = 0;
    for (int c = 1; c <= 8 && st == RSFT_OK; c <<= 1) {
      if (!rsft::fft_cluster_valid(g, c)) continue;
      for (int t : {256, 512}) {
        auto launch = [&] {
          return rsft::launch_fft_cluster(g, plan->tables, plan->ws.folded, plan->ws.spectrum, plan->ws.det_bits,
                                          plan->ws.det_count, plan->ws.words_b, true, s, 1, 0, c, t);
        };
        e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          cudaGetLastError();  // a shape the device cannot schedule: skip it
          continue;
        }
        if (ms < fft_best) {
          fft_best = ms;
          bc = c;
          bt = t;
        }
      }
    }
    plan->fft_csize = bc;
    plan->fft_threads = bt;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RSFT_OK) return st;
  if (st2 != RSFT_OK) return st2;
  if (best < 0) return fail(RSFT_ERR_UNSUPPORTED, "no candidate fold schedule could run");
  if (us_out) *us_out = best_us;
  if (chosen) *chosen = best;
  return RSFT_OK;
}

}  // extern "C"

// An execute recorded as a CUDA graph on one lane of a plan.
struct rsft_graph {
  rsft_plan* plan = nullptr;
  int lane = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

rsft_status rsft_graph_create(rsft_plan* plan, const void* d_cube, int32_t lane, uint64_t* d_located, void* d_amp,
                              int64_t* d_n_located, rsft_graph** graph) {
  if (!graph) return fail(RSFT_ERR_INVALID_ARG, "NULL graph pointer");
  *graph = nullptr;
  if (!plan || !d_cube || !d_n_located) return fail(RSFT_ERR_INVALID_ARG, "NULL plan, cube or count");
  if (!plan->has_device) return fail(RSFT_ERR_INVALID_ARG, "host-only plan cannot execute");
  if (lane < 0 || lane > 7) return fail(RSFT_ERR_INVALID_ARG, "lane must be 0..7");
  if (plan->host.desc.max_located > 0 && !d_located) return fail(RSFT_ERR_INVALID_ARG, "d_located is NULL");
  if (reinterpret_cast<uintptr_t>(d_cube) % 16 != 0) return fail(RSFT_ERR_INVALID_ARG, "cube must be 16-byte aligned");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  rsft_status st = ensure_lanes(plan, lane + 1, false);
  if (st != RSFT_OK) return st;
  rsft_lane& ln = plan->lanes[lane];
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "graph capture stream");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  bool dirty = true;  // a recorded execute always clears the vote array it starts from
  st = run_lane(plan, ln.ws, dirty, false, d_cube, cs, d_located, nullptr, static_cast<float2*>(d_amp), nullptr,
                d_n_located);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (st != RSFT_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  rsft_graph* out = new rsft_graph;
  out->plan = plan;
  out->lane = lane;
  out->graph = g;
  out->exec = x;
  *graph = out;
  return RSFT_OK;
}

rsft_status rsft_graph_create_frames(rsft_plan* plan, const void* const* d_cubes, int64_t n_frames, uint64_t* d_located,
                                     void* d_amp, int64_t* d_counts, rsft_graph** graph) {
  if (!graph) return fail(RSFT_ERR_INVALID_ARG, "NULL graph pointer");
  *graph = nullptr;
  rsft_status st = check_frames_args(plan, d_cubes, n_frames, d_located, d_counts);
  if (st != RSFT_OK) return st;
  if (n_frames < 1) return fail(RSFT_ERR_INVALID_ARG, "a frames graph needs at least one frame");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  const bool together = frames_together(plan);
  if ((st = ensure_lanes(plan, 1, false)) != RSFT_OK) return st;   // graph batches run on lane 0's stream
  if (together && (st = ensure_frames(plan)) != RSFT_OK) return st;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "graph capture stream");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  if (together) {
    st = run_frames(plan, d_cubes, n_frames, cs, d_located, static_cast<float2*>(d_amp), d_counts, false);
  } else {
    // recorded on lane 0's workspace (a recorded execute always clears its votes first)
    rsft_lane& ln = plan->lanes[0];
    const int64_t cap = plan->host.desc.max_located;
    for (int64_t f = 0; f < n_frames && st == RSFT_OK; ++f) {
      bool dirty = true;
      st = run_lane(plan, ln.ws, dirty, false, d_cubes[f], cs, d_located ? d_located + f * cap : nullptr, nullptr,
                    d_amp ? static_cast<float2*>(d_amp) + f * cap : nullptr, nullptr, d_counts + f);
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (st != RSFT_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return st;
  }
  if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  rsft_graph* out = new rsft_graph;
  out->plan = plan;
  out->lane = 0;
  out->graph = g;
  out->exec = x;
  *graph = out;
  return RSFT_OK;
}

rsft_status rsft_graph_launch(rsft_graph* graph, void* stream) {
  if (!graph || !graph->exec) return fail(RSFT_ERR_INVALID_ARG, "NULL graph");
  DeviceGuard guard(graph->plan->device);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  const cudaError_t e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? RSFT_OK : cuda_fail(e, "cudaGraphLaunch");
}

rsft_status rsft_graph_launch_batch(rsft_graph* const* graphs, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && !graphs)) return fail(RSFT_ERR_INVALID_ARG, "NULL graphs or negative count");
  if (n == 0) return RSFT_OK;
  for (int64_t i = 0; i < n; ++i)
    if (!graphs[i] || !graphs[i]->exec) return fail(RSFT_ERR_INVALID_ARG, "NULL graph in the batch");
  const int dev = graphs[0]->plan->device;
  for (int64_t i = 1; i < n; ++i)
    if (graphs[i]->plan->device != dev) return fail(RSFT_ERR_INVALID_ARG, "graphs of one batch must share a device");
  DeviceGuard guard(dev);
  if (!guard.ok) return fail(RSFT_ERR_CUDA, "cudaSetDevice failed");
  // the distinct lanes of the batch: each waits for the caller's stream, runs its graphs in
  // order, and the caller's stream waits for all of them
  std::vector<rsft_lane*> lanes;
  for (int64_t i = 0; i < n; ++i) {
    rsft_lane* ln = &graphs[i]->plan->lanes[graphs[i]->lane];
    if (std::find(lanes.begin(), lanes.end(), ln) == lanes.end()) lanes.push_back(ln);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t fork = graphs[0]->plan->fork;
  cudaError_t e = cudaEventRecord(fork, s);
  for (size_t i = 0; e == cudaSuccess && i < lanes.size(); ++i) e = cudaStreamWaitEvent(lanes[i]->stream, fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "graph batch fork");
  for (int64_t i = 0; i < n; ++i) {
    e = cudaGraphLaunch(graphs[i]->exec, graphs[i]->plan->lanes[graphs[i]->lane].stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  }
  for (size_t i = 0; e == cudaSuccess && i < lanes.size(); ++i) {
    e = cudaEventRecord(lanes[i]->done, lanes[i]->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, lanes[i]->done, 0);
  }
  return e == cudaSuccess ? RSFT_OK : cuda_fail(e, "graph batch join");
}

void rsft_graph_destroy(rsft_graph* graph) {
  if (!graph) return;
  DeviceGuard guard(graph->plan->device);
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  cudaGetLastError();
  delete graph;
}

rsft_status rsft_check_wait_timeout(int32_t limit_ms, void* stream) {
  if (limit_ms < 1 || limit_ms > 1000) return fail(RSFT_ERR_INVALID_ARG, "limit_ms must be 1..1000");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d_err = nullptr;
  cudaError_t e = cudaMalloc(&d_err, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? RSFT_ERR_OOM : RSFT_ERR_CUDA, "cudaMalloc failed");
  }
  int h_err = 0;
  e = cudaMemsetAsync(d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = rsft::launch_wait_selftest(d_err, static_cast<uint64_t>(limit_ms) * 1000000ull, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_err);
  if (e != cudaSuccess) return cuda_fail(e, "rsft_check_wait_timeout");
  if (h_err != 1) return RSFT_OK;
  return fail(RSFT_ERR_TIMEOUT, "the bounded wait gave up, as intended");
}

const char* rsft_status_string(rsft_status s) {
  switch (s) {
    case RSFT_OK: return "ok";
    case RSFT_ERR_INVALID_ARG: return "invalid argument";
    case RSFT_ERR_UNSUPPORTED: return "unsupported";
    case RSFT_ERR_OOM: return "out of memory";
    case RSFT_ERR_CAPACITY: return "output capacity exceeded";
    case RSFT_ERR_CUDA: return "CUDA error";
    case RSFT_ERR_TIMEOUT: return "device wait timed out";
    case RSFT_ERR_DESIGN: return "threshold design infeasible";
  }
  return "unknown status";
}

const char* rsft_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
