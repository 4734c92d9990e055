/*
 * rsft.h -- C ABI of the GB300 (sm_103a) RSFT hot path.
 *
 * The Realistic Sparse Fourier Transform of Wang, Patel and Petropulu ("An
 * Efficient High-Dimensional Sparse Fourier Transform"), Algorithm 1: over L
 * random loops, a windowed N-D complex cube is permuted per dimension by an
 * odd multiplier sigma (Def. 1, tau = 0 as in §III), multiplied by a flat
 * window, aliased into a B-bucket grid (Def. 2, §III-C.3), transformed by a
 * B-point N-D FFT (eq. (f)), thresholded on bucket power (first-stage
 * Neyman-Pearson detection, §IV-B eq. (tpd)), reverse-mapped into candidate
 * frequencies (Def. 4) whose votes are accumulated over loops (eq. (a_i)), and
 * thresholded again on the vote count (second stage, §III-C.5, eq. (opt)).
 * Located frequencies get a median amplitude estimate (the estimation
 * paragraph of §III).
 *
 * Conventions used by every call below:
 *  - Sizes: ndim in [1, 4]; every N_d and B_d is a power of two (§II-A
 *    notation), B_d divides N_d, N_d >= 2; M_d = N_d / B_d (the paper's L of
 *    Def. 2).  L = number of loops (the paper's T), 1..255.
 *  - Cube: complex64 (interleaved re, im float32), row-major N_0 x ... x
 *    N_{D-1}, last dimension contiguous, device memory, 16-byte aligned,
 *    owned by the caller and only read.
 *  - Linear frequency index i = sum_d i_d prod_{e>d} N_e (row-major).
 *  - Bucket index k = sum_d k_d prod_{e>d} B_e (row-major); bucket k of loop l
 *    holds the permuted bins [k_d M_d, (k_d + 1) M_d) of every dimension
 *    (the floor mapping of Def. 3).
 *  - DFTs are forward (kernel e^{-j 2 pi k n / B}) and unnormalised (eq. (f)).
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream).  Calls are stream-ordered unless stated otherwise.
 *  - Threads: a plan (its workspaces, lanes, events and the graphs recorded
 *    on it) is used by one host thread at a time; different plans may be
 *    used from different host threads at once.  The kernels' process-wide
 *    launch attributes (dynamic shared-memory limits, which are only ever
 *    raised, and cached occupancies) are set under one lock.  The one shared
 *    device array, that of rsft_stage2_static, is described there.
 *  - Errors: every call returns an rsft_status; on failure nothing is
 *    guaranteed about the outputs and rsft_last_error() holds a message.
 *    The library never traps and never falls back to the CPU: without a
 *    usable CUDA device, calls that need one return RSFT_ERR_CUDA.  Kernels
 *    wait only on their own CTA's barriers, each wait bounded (2 s); a wait
 *    that gives up sets the plan's error flag, which the synchronous calls
 *    (rsft_execute, rsft_execute_segments, rsft_execute_host,
 *    rsft_execute_host_batch) report as
 *    RSFT_ERR_TIMEOUT.
 */
#ifndef RSFT_H
#define RSFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rsft_status {
  RSFT_OK = 0,
  RSFT_ERR_INVALID_ARG = 1,   /* bad descriptor, pointer or size              */
  RSFT_ERR_UNSUPPORTED = 2,   /* valid but not implemented (e.g. ndim > 4)    */
  RSFT_ERR_OOM = 3,           /* device or host allocation failed             */
  RSFT_ERR_CAPACITY = 4,      /* output truncated; required size returned     */
  RSFT_ERR_CUDA = 5,          /* CUDA runtime error (message in last_error)   */
  RSFT_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                */
  RSFT_ERR_DESIGN = 7         /* threshold design (eq. (opt)) has no solution */
} rsft_status;

enum { RSFT_WIN_RECT = 0, RSFT_WIN_CHEB = 1 };       /* pre-permutation window (§III-A) */
enum { RSFT_FLAT_IDEAL = 0, RSFT_FLAT_CHEB = 1 };    /* flat window (§IV-B)             */
enum { RSFT_BETA_EXACT = 0, RSFT_BETA_MEAN = 1 };    /* beta(sigma_l) or beta-bar in gamma */
/* How votes are accumulated (same result): by output rows in shared memory with the
 * second stage fused (default), or by scattering every candidate of every detected
 * bucket with 8-bit atomic adds into an N-byte vote array followed by a compaction. */
enum { RSFT_VOTES_ROWS = 0, RSFT_VOTES_SCATTER = 1 };
/* Vote law of the second-stage threshold design (eq. (opt)): the Normal approximations of
 * Claims 2-3 (the paper; default), or the binomial laws they approximate.  Binomial: sigma_l
 * is drawn independently per loop (Def. 1), so a true cell's count is Binomial(L, Pd-bar)
 * and an off-target cell's Binomial(L, q), q = rho min(1, eta_p Pd-bar) + (1 - rho)
 * Pfa1-bar with rho = K_max eta_m / B (Claim 3's F / L).  The Normal form underestimates the
 * upper tail of the off-target count, where P_fa lies, so at small P_fa the binomial design
 * picks a higher mu and meets P_fa on noise; target-induced false alarms are heavier still. */
enum { RSFT_DESIGN_NORMAL = 0, RSFT_DESIGN_BINOMIAL = 1 };

/* Warning bits reported by rsft_plan_get(RSFT_GET_WARNINGS). */
enum { RSFT_WARN_SPARSITY_LIMIT = 1 };  /* K_max * eta_m >= B: Remark 2, RSFT cannot separate H0/H1 */

/*
 * Plan descriptor (Problem 1 of §IV-A: sizes, loop count, window, P_fa; the
 * Algorithm 1 inputs).  Fill with rsft_desc_init() and override fields.
 */
typedef struct rsft_desc {
  int32_t ndim;              /* D, 1..4                                               */
  int64_t n[4];              /* N_d, powers of two >= 2                               */
  int64_t b[4];              /* B_d, powers of two, B_d | N_d                          */
  int32_t loops;             /* L (paper T), 1..255                                   */
  int32_t window;            /* RSFT_WIN_CHEB (default) or RSFT_WIN_RECT              */
  double atten_db;           /* Chebyshev side-lobe attenuation in dB (default 60)    */
  int32_t flat;              /* RSFT_FLAT_CHEB (default) or RSFT_FLAT_IDEAL           */
  int64_t flat_support[4];   /* taper support S_d (even, 2..N_d); 0 = N_d             */
  double p_fa;               /* system per-bin false-alarm probability (§IV-A)       */
  double p_d;                /* system detection probability of the weakest tone     */
  int32_t k_max;             /* sparsity budget K used by the design (Claim 3)       */
  double eta_p;              /* calibration eta_p >= 1 (Claim 3); <= 0 = 1/Pd-bar     */
  double p_fa1_override;     /* > 0: first-stage Pfa1-bar; else from eq. (opt)        */
  int32_t mu_override;       /* >= 0: second-stage threshold mu; else from eq. (opt)  */
  double noise_var;          /* sigma_n^2 > 0: known noise (§IV-A).  <= 0: estimate mode:
                              * each execute takes loop l's noise floor from its own bucket
                              * powers P_l = |f-hat_l|^2 as lowermedian(P_l) / ln 2 (rank
                              * floor((B - 1) / 2) ascending; under H0 the power is
                              * exponential, eq. (exp), whose median is the mean times
                              * ln 2) and sets gamma_l = -(lowermedian(P_l) / ln 2) ln Pfa1-bar
                              * (eq. (tpd) with the estimate in place of sigma_n^2 beta)   */
  uint64_t seed;             /* SplitMix64 seed of the sigma draws                    */
  const int64_t* sigma;      /* optional [loops][ndim] odd multipliers; NULL = draw   */
  int32_t beta_mode;         /* RSFT_BETA_EXACT (default) or RSFT_BETA_MEAN           */
  int64_t max_located;       /* capacity of the located list (default 65536)          */
  int32_t device;            /* CUDA device ordinal; -1 = host-only plan (tables only) */
  int32_t vote_mode;         /* RSFT_VOTES_ROWS (default) or RSFT_VOTES_SCATTER        */
  int32_t design_mode;       /* RSFT_DESIGN_NORMAL (default) or RSFT_DESIGN_BINOMIAL   */
} rsft_desc;

typedef struct rsft_plan rsft_plan;

/* Fill *desc with defaults: ndim 0 (must be set), Chebyshev 60 dB windows,
 * p_fa 1e-6, p_d 0.9, k_max 8, eta_p 1, no overrides, noise_var 1, seed 0,
 * max_located 65536, device 0, row votes, Normal design.  desc must not be NULL. */
void rsft_desc_init(rsft_desc* desc);

/*
 * Build a plan: draw sigma (Def. 1; odd values, §V-E), build the windows
 * (§III-C.1, §IV-B), per-loop beta(sigma_l) (eq. (alpha_beta)), solve eq.
 * (opt) for (mu, Pfa1-bar) unless overridden, set gamma_l = -sigma_n^2
 * beta(sigma_l) ln Pfa1-bar (eq. (tpd)) -- or, in estimate mode (noise_var
 * <= 0), leave gamma_l to each execute (NaN in RSFT_GET_GAMMA) -- upload the
 * tables and allocate the workspace on desc->device.  With device = -1 only the host tables are
 * built (for rsft_plan_get); such a plan cannot execute.
 * Ownership: *plan is owned by the caller and released by rsft_plan_destroy.
 * Errors: INVALID_ARG (sizes, loops, windows, a non-finite noise_var, an
 * unknown design_mode), UNSUPPORTED (ndim > 4), DESIGN (no feasible mu),
 * OOM, CUDA.  On error *plan is set to NULL.
 */
rsft_status rsft_plan_create(const rsft_desc* desc, rsft_plan** plan);

/* Release a plan and its device memory (synchronises its device).  NULL is a no-op. */
void rsft_plan_destroy(rsft_plan* plan);

/*
 * Run the whole hot path on one cube (Algorithm 1 plus second-stage
 * detection and estimation) and wait for it.
 *   d_cube          device complex64 cube (see conventions).
 *   stream          cudaStream_t or NULL.
 *   d_located       device uint64 [max_located]: located linear indices,
 *                   ascending (second-stage output o of Algorithm 1).
 *   d_located_votes device uint8 [max_located] or NULL: vote count of each.
 *   d_amp           device complex64 [max_located] or NULL: median estimate of
 *                   each located amplitude (§III estimation paragraph).
 *   d_votes_out     device uint8 [N] or NULL: the accumulated votes a-bar
 *                   (eq. (a_i)) before they are cleared for the next call.
 *   n_located       host: number of located frequencies (may exceed
 *                   max_located, then RSFT_ERR_CAPACITY and the first
 *                   max_located, in ascending order, are written).
 * The plan's workspace is reused: calls on one plan must not overlap.
 */
rsft_status rsft_execute(rsft_plan* plan, const void* d_cube, void* stream,
                         uint64_t* d_located, uint8_t* d_located_votes,
                         void* d_amp, uint8_t* d_votes_out, int64_t* n_located);

/*
 * As rsft_execute, but does not wait: the located count (int64, possibly
 * above max_located) is written to device memory *d_n_located in stream
 * order, and capacity overflow is not reported as an error.  The execute's
 * kernels are launched as a programmatic-dependent chain: each may be
 * scheduled while the kernel before it on `stream` is finishing, but reads and
 * writes nothing until that kernel has completed, so stream order with respect
 * to the caller's kernels, copies and events is unchanged.
 */
rsft_status rsft_execute_async(rsft_plan* plan, const void* d_cube, void* stream,
                               uint64_t* d_located, uint8_t* d_located_votes,
                               void* d_amp, uint8_t* d_votes_out,
                               int64_t* d_n_located);

/*
 * End-to-end call on HOST buffers: copies h_cube (N complex64, preferably
 * pinned) to a plan-owned device staging buffer on `stream`, runs the hot
 * path, and copies the located list back.  h_located (uint64), h_amp
 * (complex64, may be NULL) hold max_located entries.  Synchronous.
 */
rsft_status rsft_execute_host(rsft_plan* plan, const void* h_cube, void* stream,
                              uint64_t* h_located, void* h_amp, int64_t* n_located);

/* Items of rsft_plan_get (host copies; `bytes` must be at least the size given). */
enum {
  RSFT_GET_SIGMA = 1,       /* int64 [L][D]  sigma_{l,d}                                  */
  RSFT_GET_SIGMA_INV = 2,   /* int64 [L][D]  sigma^{-1} mod N_d (eq. (mod_inv))           */
  RSFT_GET_GAMMA = 3,       /* double [L]    first-stage thresholds gamma_l               */
  RSFT_GET_BETA = 4,        /* double [L]    beta(sigma_l) (eq. (alpha_beta))            */
  RSFT_GET_MU = 5,          /* int32 [1]     second-stage threshold (votes > mu)         */
  RSFT_GET_PFA1 = 6,        /* double [1]    first-stage Pfa1-bar                        */
  RSFT_GET_ETA_M = 7,       /* double [1]    prod_d 6-dB bandwidth of w_d in bins        */
  RSFT_GET_PD_BAR = 8,      /* double [1]    Pd-bar of the design (0 if overridden)      */
  RSFT_GET_WINDOW = 9,      /* double [sum_d N_d]    pre-window taps w_d, d = 0..D-1      */
  RSFT_GET_FLAT = 10,       /* double [2 sum_d N_d]  flat-window taps (re, im) per d      */
  RSFT_GET_WARNINGS = 11,   /* int32 [1]     RSFT_WARN_* bits                            */
  RSFT_GET_SNR_DB = 12,     /* double [1]    SNR*_min of eq. (opt) in dB (half-bin tone) */
  RSFT_GET_WORKSPACE_BYTES = 13, /* int64 [1] device bytes owned by the plan              */
  RSFT_GET_STAGE_MS = 14,   /* double [8]    with timing on (rsft_plan_timing): summed device
                             * milliseconds of [0] permute_window_fold, [1] bucket_fft+np_detect,
                             * [2] vote_scatter (RSFT_VOTES_SCATTER only), [3] stage2_compact
                             * or, with RSFT_VOTES_ROWS, vote_rows, [4] median_estimate,
                             * [5] whole execute; [6] executes timed; [7] kernel launches per
                             * execute (with amplitudes).  Waits for the timed executes.      */
  RSFT_GET_FOLD_BYTES = 15, /* int64 [1]     algorithmic bytes of one execute's fold: the cube
                             * read once per loop group plus the bucket writes               */
  RSFT_GET_FOLD_COPY = 16,  /* int32 [1]     how the last fold streamed the cube: 0 one bulk copy
                             * per row, 3 or 5 one tensor-map box per stage (rank) into the SIMT
                             * fold, 103 or 105 the same boxes into the tensor-core fold (whole
                             * 64-column rows, chosen by environment RSFT_FOLD=tc at plan
                             * creation), -1 none yet                                            */
  RSFT_GET_GAMMA_LAST = 17, /* double [L]    thresholds the last execute on the plan's own
                             * workspace compared with: the plan's gamma_l with known noise, the
                             * per-loop estimates (FP32, widened) in estimate mode.  Waits for the
                             * device; NaN before the first execute in estimate mode.          */
  RSFT_GET_FRAMES_FOLD = 18,/* double [3]    with timing on: summed device milliseconds of the fold
                             * launches of rsft_execute_frames calls (not of recorded graphs), the
                             * frames they folded, and their number.  Waits for them.           */
  RSFT_GET_FFT_SHAPE = 19   /* int32 [2]     the bucket FFT's CTAs per loop (a thread-block cluster)
                             * and threads per CTA; 0, 0 when it runs as shared-memory passes     */
};
rsft_status rsft_plan_get(const rsft_plan* plan, int32_t what, void* out, size_t bytes);

/*
 * Per-stage device timing.  enable != 0 starts recording CUDA events on the
 * execute's stream around each stage (and clears the sums); 0 stops.  Read the
 * sums with rsft_plan_get(RSFT_GET_STAGE_MS).  Events add no host sync.
 */
rsft_status rsft_plan_timing(rsft_plan* plan, int32_t enable);

/* Bucket arrays of the last execute, for inspection (stream-ordered device copy). */
enum {
  RSFT_BUCKETS_FOLDED = 0,    /* f_l = Aliasing(W-bar P_sigma W r) (Algorithm 1, eq. (l)) */
  RSFT_BUCKETS_SPECTRUM = 1   /* f-hat_l = NDFFT(f_l) (eq. (f))                           */
};
/* d_out: device complex64 [L][B] (bucket k of loop l at l * B + k). */
rsft_status rsft_copy_buckets(rsft_plan* plan, int32_t which, void* d_out, void* stream);

/* First-stage detections c_l of the last execute (§IV-C): d_out device uint32
 * [L][ceil(B/32)], bit (k mod 32) of word k / 32 set iff |f-hat_l[k]|^2 > gamma_l. */
rsft_status rsft_copy_detections(rsft_plan* plan, void* d_out, void* stream);

/*
 * Refinement of off-grid tones in the bucket domain (beyond the paper, which
 * recovers grid locations only, §I).  A K-tone model s(t) = sum_k a_k
 * exp(j 2 pi f_k . t) (f_k in cycles/sample per dimension) is compared, loop by
 * loop, with the cube through the RSFT's own fold (Algorithm 1: pre-window,
 * permutation, flat window, aliasing):
 *     E = sum_l sum_j |F_l[j] - fold_l(s)[j]|^2,   F_l = fold_l(cube).
 * The fold is linear and separable over dimensions, so E, its gradient and the
 * Gauss-Newton diagonal need per-dimension tone responses only (no N-point
 * fields).  Tones: d_freq device float [K][D] (wrapped into [0, 1)), d_amp
 * device complex64 [K].
 *
 * rsft_refine_prepare: folds d_cube into the plan's buckets F_l (all loops).
 * rsft_refine_eval: E (device double *d_loss, may be NULL), dE/df (device float
 *   [K][D]), (dE/da_re, dE/da_im) as device complex64 [K], and the Gauss-Newton
 *   diagonal (device float [K][D + 1]: amplitude term, then one per frequency;
 *   NULL allowed) of the tones against the buckets of the last prepare or
 *   execute.  Stream-ordered.
 * rsft_refine: prepare, then `steps` Levenberg-Marquardt iterations, in place
 *   on d_freq and d_amp.  Each tone solves (H + lambda diag H) delta = -g with
 *   its own Gauss-Newton matrix H of (a_re, a_im, f_0 .. f_{D-1}) and moves by
 *   lr * delta; the trial is kept when the loss E drops (lambda / 10) and
 *   undone otherwise (lambda * 10), lambda starting at 1e-3.  The tones end at
 *   the kept point of lowest E (steps + 1 evaluations of E).
 * Errors: INVALID_ARG (NULL, k < 1, steps < 0, lr <= 0, misaligned cube),
 * UNSUPPORTED (K > 2^20), OOM, CUDA.
 */
rsft_status rsft_refine_prepare(rsft_plan* plan, const void* d_cube, void* stream);
rsft_status rsft_refine_eval(rsft_plan* plan, int64_t k, const float* d_freq, const void* d_amp, double* d_loss,
                             float* d_grad_freq, void* d_grad_amp, float* d_hdiag, void* stream);
rsft_status rsft_refine(rsft_plan* plan, const void* d_cube, int64_t k,
                        float* d_freq, void* d_amp, int32_t steps, float lr,
                        void* stream);

/*
 * Second-stage detection (o = {i : votes[i] > mu}, ascending) for callers that
 * cannot allocate device memory.  The paper has no counterpart: this is the
 * stage2_compact step of rsft_execute offered on its own, for code that must
 * not call cudaMalloc or cudaFree when it runs (a real-time loop whose memory
 * is fixed at start-up, a host framework that owns every allocation, code
 * that cannot afford the device synchronisation those calls may cause).
 *   d_votes          device uint8 [n], 16-byte aligned: the accumulated
 *                    per-frequency vote counts, e.g. rsft_execute's
 *                    d_votes_out.  Cleared to zero on return, as rsft_execute
 *                    clears its own votes.
 *   n                number of votes: a multiple of 16384, at most 2^28.
 *   mu               second-stage threshold, 0..254.
 *   d_located        device uint64 [capacity]: located indices, ascending.
 *   d_located_votes  device uint8 [capacity] or NULL: their vote counts.
 *   d_count          device int64 [1]: number located (may exceed capacity;
 *                    then only the first `capacity` are written).
 * Runs on the current device, stream-ordered.  It allocates nothing: its
 * scratch (per-segment counts and offsets, about 192 KiB) is a fixed array in
 * the library's device memory that every GPU loading the library holds until
 * the process exits.  The first call on a device looks that array up
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * The looked-up address is kept for the life of the process: after a device
 * reset (cudaDeviceReset, or a release and re-creation of the primary
 * context) the entry point must not be called again on that device until
 * the library is reloaded.
 * All calls share the one array: calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller.
 * Errors: INVALID_ARG for NULL pointers, misalignment, n not a multiple of
 * 16384 or above 2^28, mu out of range; CUDA for launch failures.
 */
rsft_status rsft_stage2_static(uint8_t* d_votes, int64_t n, int32_t mu, uint64_t* d_located,
                               uint8_t* d_located_votes, int64_t capacity, int64_t* d_count,
                               void* stream);

/* Segment mode (§III-C: each iteration processes its own data segment of the signal
 * model of §IV-A, with sigma_l drawn per segment): loop l folds the device cube
 * d_segments[l] (a host array of L device pointers, each 16-byte aligned, all of the
 * plan's shape); bucket FFT, detection, votes, second stage and estimate are those of
 * rsft_execute, over the L segments' buckets.  The fold reads every segment once (L
 * cubes per call).  Outputs, counts and errors as for rsft_execute / rsft_execute_async;
 * the first call builds one-loop fold tables (kept by the plan). */
rsft_status rsft_execute_segments(rsft_plan* plan, const void* const* d_segments, void* stream, uint64_t* d_located,
                                  uint8_t* d_located_votes, void* d_amp, uint8_t* d_votes_out, int64_t* n_located);
rsft_status rsft_execute_segments_async(rsft_plan* plan, const void* const* d_segments, void* stream,
                                        uint64_t* d_located, uint8_t* d_located_votes, void* d_amp,
                                        uint8_t* d_votes_out, int64_t* d_n_located);

/*
 * Frames of this plan's shape in one launch per stage: the fold of up to 16
 * frames is one persistent launch whose work units run over (frame, unit),
 * each frame's cube with its own tensor map; the bucket FFT, the detection,
 * the vote count, the second stage and the median estimate each take all those
 * frames' loops in one launch (frames along the grid's second dimension).
 * Larger counts go in groups of 16.  Frame f reads d_cubes[f] (a host array of
 * device pointers, each 16-byte aligned), writes its located list to d_located +
 * f * max_located (ascending), its amplitudes (when d_amp is not NULL) to d_amp +
 * f * max_located, and its located count to d_counts[f] (device int64; above
 * max_located means the list was truncated).  Stream-ordered, no host
 * synchronisation, results identical to one rsft_execute_async per frame.  The
 * first call allocates the frames' workspace (kept by the plan), so make it
 * before any stream capture; calls on one plan must not overlap.  Plans whose
 * stages cannot take several frames (rsft_plan_frames_together gives 0: a
 * chunked or tensor-core fold, loops in several passes, shared-memory FFT
 * passes, scatter votes) run the frames one after another instead.  The paper
 * processes one cube at a time and has no counterpart.
 * Errors: INVALID_ARG (NULL pointers, n_frames < 0, a misaligned cube), OOM, CUDA.
 */
rsft_status rsft_execute_frames(rsft_plan* plan, const void* const* d_cubes, int64_t n_frames, void* stream,
                                uint64_t* d_located, void* d_amp, int64_t* d_counts);
/* *together = 1 when rsft_execute_frames runs this plan's frames together, else 0. */
rsft_status rsft_plan_frames_together(const rsft_plan* plan, int32_t* together);

/* Batched executes of n_frames equally shaped device cubes (this plan's shape):
 * frame f reads d_cubes[f] (a host array of device pointers, each 16-byte
 * aligned), writes its located list to d_located + f * max_located, its
 * amplitudes (when d_amp is not NULL) to d_amp + f * max_located, and its full
 * located count to d_counts[f] (device int64).  Frames go round-robin to
 * `lanes` execution lanes (1..8), each with its own workspace (created on
 * first use, kept by the plan) and stream.  The lanes start after the work
 * already queued on `stream`, and `stream` waits for all of them, so the call
 * is stream-ordered like rsft_execute_async; concurrent lanes overlap one
 * frame's fold with another frame's bucket FFT, votes and estimate.  Per-frame
 * stage timing is not recorded.  The paper has no counterpart (it processes one
 * cube at a time).  Errors: INVALID_ARG (NULL pointers, n_frames < 0, lanes
 * outside 1..8, a misaligned cube), OOM, CUDA. */
rsft_status rsft_execute_batch(rsft_plan* plan, const void* const* d_cubes, int64_t n_frames, int32_t lanes,
                               void* stream, uint64_t* d_located, void* d_amp, int64_t* d_counts);

/* CUDA-graph form of an execute.  rsft_graph_create records, by stream capture, the
 * launches rsft_execute_async makes for one cube and one set of outputs on execution
 * lane `lane` (0..7, the lanes of rsft_execute_batch: each its own workspace and
 * stream, created on first use) and instantiates them.  The pointers are fixed in the
 * graph: every launch re-reads d_cube (device, 16-byte aligned, the plan's N complex64)
 * and rewrites d_located (device uint64 [max_located]), d_amp (device complex64
 * [max_located] or NULL) and d_n_located (device int64 [1]).  Graphs on one lane share
 * its workspace, so the caller orders them (rsft_graph_launch_batch runs each lane's
 * graphs in order on the lane's stream).  A graph keeps the plan's fold schedule and
 * tables of the moment it was recorded: re-record after rsft_plan_autotune, and destroy
 * every graph before its plan.  The paper has no counterpart.
 * Errors: INVALID_ARG (NULL pointers, lane outside 0..7, misaligned cube), OOM, CUDA. */
typedef struct rsft_graph rsft_graph;
rsft_status rsft_graph_create(rsft_plan* plan, const void* d_cube, int32_t lane, uint64_t* d_located, void* d_amp,
                              int64_t* d_n_located, rsft_graph** graph);
/* One launch of a recorded execute on `stream` (cudaGraphLaunch).  Errors: INVALID_ARG, CUDA. */
/* rsft_execute_frames of n_frames cubes recorded as one CUDA graph (results to
 * d_located / d_amp / d_counts as there); launched like any other graph of this
 * plan, on the stream of its lane 0.  The paper has no counterpart. */
rsft_status rsft_graph_create_frames(rsft_plan* plan, const void* const* d_cubes, int64_t n_frames,
                                     uint64_t* d_located, void* d_amp, int64_t* d_counts, rsft_graph** graph);
rsft_status rsft_graph_launch(rsft_graph* graph, void* stream);
/* A batch of recorded executes, possibly of different plans (frames of different shapes):
 * the lanes the graphs belong to start after the work queued on `stream`, each runs its
 * graphs in the order given on its own stream, and `stream` waits for all of them.
 * All graphs must be on one device.  Errors: INVALID_ARG (NULL graph, n < 0, mixed
 * devices), CUDA. */
rsft_status rsft_graph_launch_batch(rsft_graph* const* graphs, int64_t n, void* stream);
void rsft_graph_destroy(rsft_graph* graph);

/* Fold-schedule autotuner.  The plan's fold schedule (which dimensions index rows and
 * which columns, how many residue classes a unit holds side by side, rows per step) comes
 * from a cost model; this call times the model's `candidates` best schedules (1..16) on
 * the caller's cube -- two warm-up and `reps` (1..1000) timed fold launches each, CUDA
 * events on `stream` -- and keeps the fastest, rebuilding the plan's fold tables.
 * d_cube: device, 16-byte aligned, the plan's N complex64 (only its timing matters).
 * *us_out (may be NULL): the winner's microseconds per fold launch; *chosen (may be NULL):
 * its rank among the candidates (0 = the model's choice).  With the cluster FFT it then
 * times every valid shape of the bucket FFT (CTAs per loop 1, 2, 4 or 8, i.e. buckets per
 * CTA, and 256 or 512 threads per CTA) on the cube's buckets and keeps the fastest
 * (RSFT_GET_FFT_SHAPE).  Results of executes do not depend on the schedule beyond FP32
 * summation order; the FFT's shape does not change its arithmetic.  Synchronises `stream`; not to be
 * called while the plan executes on another stream.  The paper has no counterpart.
 * Errors: INVALID_ARG, UNSUPPORTED (no candidate could run), OOM, CUDA. */
/* Shape of the bucket FFT's cluster launch: ctas_per_loop CTAs (1, 2, 4 or 8; each holds
 * B / ctas_per_loop buckets of a loop) of `threads` threads (256 or 512); 0, 0 restores the
 * default.  The arithmetic does not depend on the shape.  Errors: INVALID_ARG, UNSUPPORTED
 * (shared-memory FFT passes, or a shape the bucket grid does not allow). */
rsft_status rsft_plan_set_fft_shape(rsft_plan* plan, int32_t ctas_per_loop, int32_t threads);

rsft_status rsft_plan_autotune(rsft_plan* plan, const void* d_cube, void* stream, int32_t candidates, int32_t reps,
                               double* us_out, int32_t* chosen);

/* Loops folded per pass over the cube (1..16; a new plan folds up to 16 loops per pass, so
 * the radar and mixed-size cubes are read once per execute).  Fewer loops per pass read the
 * cube ceil(L / loops_per_pass) times with less arithmetic per byte in each pass: the
 * trade-off between one fused, compute-bound pass and several HBM-bound ones (results are
 * the same up to FP32 summation order).  Rebuilds the plan's fold tables after waiting for
 * the device; graphs recorded before must be recorded again.  The paper has no counterpart
 * (Algorithm 1 folds each loop on its own).  Errors: INVALID_ARG (NULL or host-only plan,
 * value outside 1..16), UNSUPPORTED, OOM, CUDA. */
rsft_status rsft_plan_set_loops_per_pass(rsft_plan* plan, int32_t loops_per_pass);

/* Host-buffer batch: frame f reads the host cube h_cubes[f] (pinned memory gets
 * the full copy bandwidth).  Returns when every frame's results are in host
 * memory: h_counts[f] (full count), the first min(count, max_located) entries
 * of h_located + f * max_located and (when h_amp is not NULL) of
 * h_amp + f * max_located.  Two lanes alternate so that the host-to-device copy
 * of frame f + 1 overlaps the RSFT of frame f; each lane keeps a device cube
 * buffer.  CAPACITY when some count exceeds max_located; TIMEOUT when a device
 * wait gave up.  The paper has no counterpart. */
rsft_status rsft_execute_host_batch(rsft_plan* plan, const void* const* h_cubes, int64_t n_frames, void* stream,
                                    uint64_t* h_located, void* h_amp, int64_t* h_counts);

/* ---------------------------------------------------------------------------
 * Dense comparison detector: the Bartlett method of Appendix A (Algorithm 2)
 * with one data segment.  The whole cube is windowed with the same pre-window
 * as the RSFT (product of the per-dimension windows, §III-C), transformed by
 * the full N-point N-D FFT (forward, unnormalised) and every bin's power is
 * tested against the exact one-segment Neyman-Pearson threshold
 *     gamma = -sigma_n^2 ||w||^2 ln P_fa
 * (under H0 the bin power is exponential with mean sigma_n^2 ||w||^2).
 * Detected bins are returned in ascending row-major order with the amplitude
 * estimate u-hat_k / prod_d sum_t w_d(t) (the amplitude of an on-grid tone).
 * The FFT is cuFFT's; windowing, power, threshold and the ordered compaction
 * are this library's kernels.
 */
typedef struct rsft_bartlett_plan rsft_bartlett_plan;

/* Plan for the dense detector.  Uses desc->ndim, n, window, atten_db, p_fa,
 * noise_var, max_located and device (b, loops and the RSFT design fields are
 * ignored).  Owns the windowed-spectrum buffer (8 N bytes), cuFFT's plan and
 * workspace.  Errors: INVALID_ARG (NULL, n not a power of two, ndim out of
 * 1..4, p_fa outside (0, 1), noise_var <= 0), UNSUPPORTED (more than 2^31 - 1
 * points), OOM, CUDA (cuFFT plan failure). */
rsft_status rsft_bartlett_plan_create(const rsft_desc* desc, rsft_bartlett_plan** plan);

/* Frees the plan and its device memory (NULL is a no-op). */
void rsft_bartlett_plan_destroy(rsft_bartlett_plan* plan);

/* One dense detection of the device cube d_cube (complex64, row-major,
 * 16-byte aligned, not modified) on `stream`.  Writes at most max_located
 * ascending detected linear indices to d_located and, when d_amp is not NULL,
 * their amplitudes (complex64) to d_amp.  *n_located (host) receives the full
 * count after a synchronisation of `stream`; CAPACITY when it exceeds
 * max_located (the outputs hold the first max_located). */
rsft_status rsft_bartlett_execute(rsft_bartlett_plan* plan, const void* d_cube, void* stream, uint64_t* d_located,
                                  void* d_amp, int64_t* n_located);

/* Stream-ordered variant: the full count lands in device memory (*d_n_located). */
rsft_status rsft_bartlett_execute_async(rsft_bartlett_plan* plan, const void* d_cube, void* stream,
                                        uint64_t* d_located, void* d_amp, int64_t* d_n_located);

/* Plan items: GAMMA (double, the threshold), GAIN (double, prod_d sum_t w_d),
 * WINDOW (double[sum_d N_d], the per-dimension windows), WORKSPACE_BYTES (int64). */
enum {
  RSFT_BARTLETT_GAMMA = 1,
  RSFT_BARTLETT_GAIN = 2,
  RSFT_BARTLETT_WINDOW = 3,
  RSFT_BARTLETT_WORKSPACE_BYTES = 4
};
rsft_status rsft_bartlett_get(const rsft_bartlett_plan* plan, int32_t what, void* out, size_t bytes);

/* Copies the last execute's spectrum (N complex64, row-major) to d_out. */
rsft_status rsft_bartlett_copy_spectrum(const rsft_bartlett_plan* plan, void* d_out, void* stream);

/*
 * Check of the bounded device waits (the paper has no counterpart).  Every wait of the
 * library's kernels on a barrier gives up after a time limit, sets an error flag and lets
 * its kernel return (see Errors above).  This call runs one CTA that waits, through the same
 * device routine as the fold, on a barrier that nothing ever completes, with a limit of
 * limit_ms milliseconds (1..1000).  It returns RSFT_ERR_TIMEOUT when the wait gave up and
 * reported it -- the expected result -- and leaves the device context usable.
 * Synchronous on `stream` (current device).  Errors: INVALID_ARG (limit out of range), OOM,
 * CUDA; RSFT_OK would mean the wait did not report giving up.
 */
rsft_status rsft_check_wait_timeout(int32_t limit_ms, void* stream);

/* Static description of a status code (never NULL). */
const char* rsft_status_string(rsft_status status);

/* Message of the last failing call on this thread ("" if none; never NULL). */
const char* rsft_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RSFT_H */
