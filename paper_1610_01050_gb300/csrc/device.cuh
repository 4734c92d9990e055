// Device-side geometry, schedules and kernel launchers of the RSFT hot path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsft {

// Programmatic dependent launch along an execute's chain of kernels (fold, FFT, vote count,
// emit, median): a kernel launched with launch_chained may be scheduled while the kernel before
// it on the stream is still finishing.  Every chained kernel calls chain_wait() before it reads
// or writes anything (it returns once the previous grid has completed and its memory is
// visible), then chain_release() so that its own successor can start launching; launched
// without the attribute, both are no-ops.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void chain_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Whether this host thread's launches through launch_chained (and the cluster FFT) carry the
// attribute.  The frames form turns it off while it launches: there two plans' groups run on
// two streams, and a chained kernel's CTAs, resident early and waiting on their predecessor,
// would hold SMs that the other stream's kernels could use (16-frame groups of the radar cube:
// 25.5k against 24.2k frames/s in the two-plan form).
inline thread_local bool t_chain_launches = true;
struct ChainLaunches {  // scope that sets the flag and restores it
  bool saved;
  explicit ChainLaunches(bool on) : saved(t_chain_launches) { t_chain_launches = on; }
  ~ChainLaunches() { t_chain_launches = saved; }
};

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                           Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = t_chain_launches ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

constexpr int kMaxDim = 4;
constexpr int kMaxLoopGroup = 16;    // loops folded per pass over the cube
constexpr int kFoldConsumers = 256;  // fold consumer threads per CTA (two columns each)
constexpr int kMaxFrames = 16;       // frames of one plan processed by one launch per stage

// Sizes of the cube and the bucket grid, in the form the kernels index with.
struct Geometry {
  int ndim;
  int loops;
  int64_t n[kMaxDim];
  int64_t b[kMaxDim];
  int64_t m[kMaxDim];
  int log_n[kMaxDim];
  int log_b[kMaxDim];
  int log_m[kMaxDim];
  int64_t total_n;
  int64_t total_b;
  int n_shift[kMaxDim];   // log2 of prod_{e>d} N_e (linear frequency index)
  int b_shift[kMaxDim];   // log2 of prod_{e>d} B_e (linear bucket index)
};

// How the fold splits the cube: dimensions [0, d_in) index rows, [d_in, D) columns.
// A CTA owns one outer residue class (x_e = s_e mod B_e, e < d_in), one chunk of that
// class's rows and one chunk of W columns; each thread keeps two fixed columns.
struct FoldSchedule {
  int d_in;               // first inner (column) dimension
  int64_t row_len;        // prod_{e >= d_in} N_e
  int width;              // W: columns per chunk (power of two, divides 2 * threads)
  int col_chunks;         // row_len / W
  int classes;            // prod_{e < d_in} B_e
  int rows_per_class;     // prod_{e < d_in} M_e
  int rows_per_chunk;     // rows of each class per unit
  int row_chunks;
  int xcount;             // X: inner residues per chunk = prod_{e >= d_in} B_e
  int direct;             // 1: one chunk per class, write buckets directly
  int cps;                // C: residue classes side by side in a row step (consecutive x_{d_in - 1})
  int crow;               // rows of each class per row step (C * crow * W <= 2 * threads)
  int groups;             // classes / C
  int red_mask;           // lane bits whose flip keeps a thread's (class, column residue) (shuffle-summed)
  int leaders;            // lanes per warp left after the shuffle sum: 32 >> popcount(red_mask)
  int slots_per_x;        // epilogue partial sums per (class, residue): 2 * warps * leaders / (C X)
  unsigned lane_perm;     // thread -> column pair: nibble b is the pair-index bit that thread bit b sets
};

// Column pair (float4 index into a row step) of fold thread tid: the thread's bits placed as
// lane_perm says (the identity 0x76543210 is the pair tid itself).
__host__ __device__ __forceinline__ int fold_pair_of(int tid, unsigned lane_perm) {
  int q = 0;
#pragma unroll
  for (int b = 0; b < 8; ++b) q |= ((tid >> b) & 1) << ((lane_perm >> (4 * b)) & 15u);
  return q;
}

// Row steps (2 * kFoldConsumers elements each) per stage of the fold's shared-memory ring: every
// whole stage of a unit is a run of this many steps (fewer when the unit's rows are fewer).
constexpr int kFoldStepsPerStage = 8;
__host__ __device__ __forceinline__ int fold_stage_steps(const FoldSchedule& fs) {
  const int steps = fs.rows_per_chunk / fs.crow;
  return steps < kFoldStepsPerStage ? steps : kFoldStepsPerStage;
}

// Fold row-table record of one (row, class) for a group of lg loops (float4 units): ceil(lg / 2)
// float4 holding the pairs (d - c, c + d) of two loops each, then ceil(lg / 4) float4 holding c of
// four loops each (w = c + jd the loop's row weight; entries past lg are zero).
__host__ __device__ __forceinline__ constexpr int fold_record_f4(int lg) { return (lg + 1) / 2 + (lg + 3) / 4; }

// One FFT pass over the bucket arrays: transforms dimensions [da, db) in shared memory.
struct FftPass {
  int da, db;
  int64_t group;          // prod_{da <= d < db} B_d
  int64_t inner;          // prod_{d >= db} B_d
  int64_t outer;          // prod_{d < da} B_d
  int64_t width;          // W consecutive inner indices per slab
  int64_t outer_per_cta;  // consecutive outer indices per CTA (when width == inner)
  int64_t ctas_per_loop;
  int last;               // final pass: writes the spectrum and the detections
};

// Row-organised vote counting: trailing dimensions [d_v, D) form a row of n_in
// locations whose buckets lie in one plane of b_in buckets per loop.
struct VoteRowSchedule {
  int d_v;
  int64_t n_in;        // prod_{e >= d_v} N_e
  int b_in;            // prod_{e >= d_v} B_e
  int m_in;            // prod_{e >= d_v} M_e
  int64_t rows;        // N / n_in
  int rows_per_warp;
  int64_t warps;       // ceil(rows / rows_per_warp)
  int small;           // rows of <= 64 locations: bit-sliced lane-per-row counting
};

// Device pointers and tables owned by a plan.
struct DeviceTables {
  const float2* wtab[kMaxDim];   // [L][N_d]: w-bar_d(sigma^{-1} s mod N_d) * w_d(s)
  const float2* wcls[kMaxDim];   // [B_d][L][M_d]: the same weights grouped by residue x = s mod B_d
  const int* sigma;              // [L][D]
  const int* sigma_inv;          // [L][D] mod N_d
  const int* sigma_inv_b;        // [L][D] sigma^{-1} mod B_d
  const float* gamma;            // [L]
  const float2* twiddle[kMaxDim];// [B_d / 2]: e^{-j 2 pi k / B_d}
  const float2* ginv[kMaxDim];   // [M_d]: 1 / G_d(-v) (dimension 0 also holds 1 / sum w)
  const unsigned short* slots_by_x; // [X][slots_per_x]: epilogue partial sums of each residue
  const float4* ftable;          // fold row table [loop group][class group][row chunk][stage][row slot][step][record]
                                 // (fold_record_f4: (d-c, c+d) pairs, then c values)
  int64_t ftable_group_f4;       // float4 of the row table per full loop group
  int ftable_group;              // loops per group the row table was built for
  const float2* fcolw;           // fold column weights [loop group][col chunk][lg][W]
  const int* h_sinvb;            // host copies of small tables passed as kernel parameters
  const unsigned short* h_slots;
  const unsigned short* h_xdig;
  const unsigned short* x_digits;   // [X][4]: inner residue digit per inner dimension
  const uint64_t* rowmask;          // rows <= 64: per loop, the candidate mask of every detection pattern of a
                                    // plane ([L][2^b_in], b_in <= 8) or of each inner bucket ([L][b_in])
  const uint16_t* kb16;             // per row dimension d < d_v: [N_d][L rounded up to 8] bucket offset (Def. 3) of index i_d
  const unsigned char* h_xres;      // host: residue index of each column of a 64-column chunk
};

struct Workspace {
  float2* folded;        // [L][B]   f_l (paper order)
  float2* spectrum;      // [L][B]   f-hat_l
  float2* partial;       // [L][classes][chunks][X] fold partial sums (chunked schedules)
  uint32_t* det_bits;    // [L][words_b]
  uint32_t* det_count;   // [L]
  uint32_t* votes;       // [ceil(N / 16) * 4] packed 8-bit votes
  uint32_t* seg_count;   // [segments] stage-2 hits per segment
  uint64_t* seg_offset;  // [segments + 1] exclusive scan of seg_count; last = total
  int* err_flag;         // set by a bounded device wait that gave up
  float* gamma_used;     // [L] first-stage thresholds of the last execute (estimate mode)
  uint32_t* warp_count;  // [row warps] vote_rows hits per warp
  uint64_t* warp_offset; // [row warps + 1]
  ulonglong2* row_list;  // small-row vote kernel: per warp [rows_per_warp] (row, votes > mu mask)
  uint32_t* warp_rows;   // [row warps] entries of each warp's row list
  int64_t words_b;
  int64_t segments;
  int64_t vote_words;
};

// Bucket-domain refinement: geometry and scratch (see refine.cu).
struct RefineGeom {
  int ndim, loops;
  int64_t n[kMaxDim], b[kMaxDim], m[kMaxDim];
  int b_shift[kMaxDim];
  int boff[kMaxDim];  // offset of dimension d in a tone's sum_d B_d responses
  int sumb;
  int64_t total_b;
};

struct RefineWork {
  float2* gres = nullptr;   // [L][K][sum B_d] per-dimension tone responses g
  float2* gder = nullptr;   // [L][K][sum B_d] their frequency derivatives g'
  float2* resid = nullptr;  // [L][B] residual buckets, source residue order
  double* partial = nullptr;
  int parts = 0;            // residual blocks (loss partial sums)
  float* contr = nullptr;   // [L][K][3 + 5 kMaxDim + kMaxDim (kMaxDim - 1)] contractions
  double* lm_gh = nullptr;  // [2][K][kLmTone] g and Gauss-Newton matrix per tone: last trial, accepted point
  float* lm_freq = nullptr; // [K][D] frequencies of the accepted point
  float2* lm_amp = nullptr; // [K] amplitudes of the accepted point
  double* lm_state = nullptr;  // [2][E, lambda] (one half per iteration), [4] E of the last trial
  int64_t k_cap = 0;
};
constexpr int kLmTone = (kMaxDim + 2) + (kMaxDim + 2) * (kMaxDim + 2);

// Launchers (return cudaSuccess or the launch error).
// Loss, gradient and Gauss-Newton diagonal of K tones against the folded buckets (each may be
// null); with gh set, each tone's gradient and Gauss-Newton matrix are stored there too.
cudaError_t launch_refine_eval(const RefineGeom& rg, const DeviceTables& t, const RefineWork& w,
                               const float2* folded, int K, const float* freq, const float2* amp, double* loss,
                               float* grad_freq, float2* grad_amp, float* hdiag, double* gh, cudaStream_t stream);
// One Levenberg-Marquardt iteration (iter = 0, 1, ...): evaluate the tones' current parameters,
// accept or reject them against the accepted point's loss (adapting the damping), and move the
// tones to the next trial -- or, with final_call, back to the accepted point.
cudaError_t launch_refine_step(const RefineGeom& rg, const DeviceTables& t, const RefineWork& w,
                               const float2* folded, int K, float* freq, float2* amp, int iter, float lr,
                               bool final_call, cudaStream_t stream);
// Exclusive scan of n u32 counts into offsets[0..n] (offsets[n] = total), total also to *total.
cudaError_t launch_count_scan(const uint32_t* counts, int64_t n, uint64_t* offsets, int64_t* total,
                              cudaStream_t stream);
// Two word ranges the fold zeroes on its way (the detection bitmaps and counts that the bucket
// FFT then fills), so an execute needs no separate clearing launches.
struct FoldClear {
  uint32_t* a = nullptr;
  int64_t na = 0;
  uint32_t* b = nullptr;
  int64_t nb = 0;
};
cudaError_t launch_fold(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t,
                        const float2* cube, int loop0, int lg, float2* folded, float2* partial, int* err,
                        int* copy_mode, cudaStream_t stream, const FoldClear& clear = FoldClear{});
// The fold of `nframes` cubes of one plan in one persistent launch (direct schedules): frame f's
// buckets go to folded + f * folded_stride.
cudaError_t launch_fold_frames(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t,
                               const float2* const* cubes, int nframes, int64_t folded_stride, int loop0, int lg,
                               float2* folded, float2* partial, int* err, int* copy_mode, cudaStream_t stream,
                               const FoldClear& clear = FoldClear{});
cudaError_t launch_fold_reduce(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t,
                               int loop0, int lg, const float2* partial, float2* folded,
                               cudaStream_t stream);
cudaError_t launch_fft_pass(const Geometry& g, const FftPass& ps, const DeviceTables& t,
                            const float2* in, float2* out, uint32_t* det_bits, uint32_t* det_count,
                            int64_t words_b, bool detect, cudaStream_t stream);
// The whole N-D bucket FFT of every loop in one launch: C CTAs per loop in a thread-block cluster
// (fft_cluster_size: 0 when the bucket grid does not allow it), detection fused when `detect`.
int fft_cluster_size(const Geometry& g);
bool fft_cluster_valid(const Geometry& g, int csize);
// With nframes > 1 the arrays hold frames one after another ([frame][L][B] buckets, [frame][L] counts,
// frame_bits detection words per frame).  csize / threads 0 take the default shape (about 2048
// buckets per CTA; 512 threads from 2048 buckets per CTA, else 256).
// gamma_out non-null: estimate mode fused in (each loop's threshold from its own lower-median bucket
// power times floor_factor, written to gamma_out[frame][l], then its detections); detect must be false.
cudaError_t launch_fft_cluster(const Geometry& g, const DeviceTables& t, const float2* in, float2* out,
                               uint32_t* det_bits, uint32_t* det_count, int64_t words_b, bool detect,
                               cudaStream_t stream, int nframes = 1, int64_t frame_bits = 0, int csize = 0,
                               int threads = 0, float* gamma_out = nullptr, float floor_factor = 0.f);
// Estimate mode of the first stage: per loop, gamma_l = lowermedian(|f-hat_l|^2) * factor (written to
// gamma_out[l]) and the loop's detection bitmap and count against it.
cudaError_t launch_noise_floor(const Geometry& g, const float2* spectrum, float factor, float* gamma_out,
                               uint32_t* det_bits, uint32_t* det_count, int64_t words_b, cudaStream_t stream,
                               int nframes = 1, int64_t frame_bits = 0);
cudaError_t launch_vote_scatter(const Geometry& g, const DeviceTables& t, const uint32_t* det_bits,
                                int64_t words_b, uint32_t* votes, cudaStream_t stream);
cudaError_t launch_stage2(const Geometry& g, int mu, Workspace& ws, uint64_t* located,
                          uint8_t* located_votes, uint8_t* votes_out, int64_t capacity,
                          int64_t* d_count, cudaStream_t stream);
cudaError_t launch_median(const Geometry& g, const DeviceTables& t, const float2* spectrum,
                          const uint64_t* located, const int64_t* d_count, int64_t capacity,
                          float2* amp, cudaStream_t stream, int nframes = 1);
int64_t stage2_segments(int64_t total_n);   // 16 KiB vote segments covering N bytes
cudaError_t launch_vote_rows(const Geometry& g, const VoteRowSchedule& vs, const DeviceTables& t,
                             const uint32_t* det_bits, int64_t words_b, int mu, uint32_t* warp_count,
                             uint64_t* warp_offset, uint64_t* located, uint8_t* located_votes,
                             uint8_t* votes_out, int64_t capacity, int64_t* d_count, int* err,
                             ulonglong2* row_list, uint32_t* warp_rows, cudaStream_t stream, int nframes = 1,
                             int64_t frame_bits = 0);
// Shared memory and resident blocks per SM of the small-row vote kernel.
size_t vote_rows_small_smem(const Geometry& g, const VoteRowSchedule& vs, int64_t words_b);
cudaError_t vote_rows_small_residency(const Geometry& g, const VoteRowSchedule& vs, int64_t words_b,
                                      int* warps_per_sm);

int fold_smem_bytes(const Geometry& g, const FoldSchedule& fs, int lg);
// One CTA waits on a barrier that never completes, through the fold's bounded wait with the
// given limit; *err is set to 1 when the wait gives up.
cudaError_t launch_wait_selftest(int* err, uint64_t limit_ns, cudaStream_t stream);

// Tensor-core fold (fold_tc.cu): schedules with 64-column chunks, two or more classes side
// by side, whole classes, rows in stages of 16.
bool fold_tc_supported(const Geometry& g, const FoldSchedule& fs);
cudaError_t launch_fold_tc(const Geometry& g, const FoldSchedule& fs, const DeviceTables& t, const float2* cube,
                           int loop0, int lg, float2* folded, int* err, int* copy_mode, cudaStream_t stream);

// Process-wide launch attributes, safe from several host threads: raise a kernel's dynamic
// shared-memory limit on the current device to at least `bytes` (never lowered, so a launch on
// another thread that relied on a higher limit stays valid), and the number of CTAs of `threads`
// threads with `bytes` of dynamic shared memory that fit on the whole current device (cached
// per device, kernel and size).  Both take one mutex.
cudaError_t ensure_smem_limit(const void* func, int bytes);
cudaError_t device_resident_ctas(const void* func, int threads, int bytes, int* ctas);

// Message returned by rsft_last_error() on this thread.
void set_last_error(const char* msg);

}  // namespace rsft
