/*
 * nfhmm.h -- C ABI of the GB300 (sm_103a) library for variational inference
 * in the Bayesian non-negative factorial HMM (N-FHMM) of Mysore & Sahani,
 * "Variational Inference in Non-negative Factorial Hidden Markov Models for
 * Efficient Audio Source Separation" (ICML 2012).
 *
 * The library computes, on one GPU, the sweep of Section 3.2:
 *   Eq. 6   alpha_tk = sum_l V_lt z_tlk + gamma sum_s sum_n d_tn^(s) B_snk + 1
 *   Eq. 7   log z_tlk = log beta_l(k) + psi(alpha_tk) - psi(sum_k alpha_tk) - kappa
 *   Eq. 8   phi_tn^(s) = gamma sum_k B_snk (psi(alpha_tk) - psi(sum_k alpha_tk))
 *   forward-backward on each source's chain with emissions exp(phi^(s))
 * plus the variational lower bound and the separation of Section 4.
 *
 * Conventions shared by every call
 * --------------------------------
 * Sizes: S sources, N states (dictionaries) per source, K elements per
 * dictionary, M = S*N*K elements, F frequency bins, T frames.  Element index
 * k = (s*N + n)*K + j: the mask B_snk of Section 2.2 is implicit (block
 * (s, n) is the K consecutive elements starting at (s*N + n)*K).
 * Layouts are row-major, C order:
 *   V     T x F    spectrogram, V[t*F + l] = V_lt >= 0 (quanta may be fractional)
 *   W     M x F    dictionary elements, W[k*F + l] = beta_l(k); each row sums to 1
 *   A     S x N x N  A[(s*N + i)*N + j] = P(D_t = j | D_{t-1} = i), rows sum to 1
 *                  (the paper's rho^(s) holds the same numbers by columns, Sec. 2.1)
 *   pi    S x N    initial state distributions, rows sum to 1
 *   dhat  S x T x N  state marginals d-hat_tn^(s) of q(D^(s))
 *   alpha T x M    Dirichlet parameters alpha-hat_tk of q(theta_t)
 *   counts T x M   sum_l V_lt z-hat_tlk (first term of Eq. 6)
 *   out   S x T x F  separated spectrograms
 * Ownership: the caller owns every buffer it passes; the library copies what
 * it keeps.  A context owns its device memory until nfhmm_destroy.
 * Pointers flagged "on device" are CUDA device pointers of the current
 * device; otherwise they are host pointers (pinned or pageable).  Spectrograms
 * in device memory or in mapped pinned host memory are read in place by a
 * kernel (over the host link for host memory); pageable ones are copied.
 * Streams: a context orders all its work after the work already queued on
 * the stream given to nfhmm_vi_init, and the stream waits for the context's
 * work before anything queued later.  Calls return once the work is queued,
 * except calls that write host memory or return a bound, which synchronise.
 * Errors: every int-returning call returns NFHMM_OK (0) or a negative code;
 * nfhmm_last_error() gives a message for the calling thread's last failure.
 * A call that fails validation leaves the context unchanged.  Every call
 * accepts a NULL context and returns NFHMM_EINVAL.
 */
#ifndef NFHMM_H
#define NFHMM_H

#include <stddef.h>

#if defined(__GNUC__)
#define NFHMM_API __attribute__((visibility("default")))
#else
#define NFHMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define NFHMM_OK        0
#define NFHMM_EINVAL   (-1)  /* bad sizes, NULL pointers, invalid inputs      */
#define NFHMM_ENOMEM   (-2)  /* device allocation failed                      */
#define NFHMM_ECUDA    (-3)  /* a CUDA call failed                            */
#define NFHMM_ETIMEOUT (-4)  /* a bounded device wait gave up                 */
#define NFHMM_ENUMERIC (-5)  /* reconstruction vanished where V > 0, or NaN   */
#define NFHMM_ESTATE   (-6)  /* call needs a state the context does not have  */
#define NFHMM_EFULL    (-7)  /* a batch has no room (frames or job slots)     */

#define NFHMM_FP32      0  /* contractions on tcgen05 tensor cores in split TF32 (FP32 accuracy) */
#define NFHMM_BF16      1  /* contractions on tcgen05 tensor cores, BF16 operands, FP32 accumulate */
#define NFHMM_FP32_SIMT 2  /* contractions on CUDA cores in FP32 (the plain GPU path)            */

#define NFHMM_INIT_UNIFORM 0  /* d-hat = 1/N                 */
#define NFHMM_INIT_PRIOR   1  /* d-hat = pi A^t (prior marginals) */

#define NFHMM_SEP_MEAN        0  /* weights v_t alpha_tk / sum_k alpha_tk (posterior mean) */
#define NFHMM_SEP_EXPECTATION 1  /* weights exp(psi(alpha_tk)), the weights of Eq. 7      */

typedef struct nfhmm_ctx nfhmm_ctx;

typedef struct {
  int S, N, K, F, T;  /* all >= 1                                          */
  double gamma;       /* Dirichlet concentration of Eq. 1 (paper: 1), >= 0 */
  int precision;      /* NFHMM_FP32, NFHMM_BF16 or NFHMM_FP32_SIMT         */
  int init_mode;      /* NFHMM_INIT_UNIFORM or NFHMM_INIT_PRIOR            */
} nfhmm_dims;

/*
 * nfhmm_vi_init -- create a context for one spectrogram (Section 3.2).
 * Copies V, W, A, pi into device memory, validates them (V finite and >= 0;
 * W, A, pi non-negative with rows summing to 1 within 1e-4) and sets the
 * initial state: z-hat from equal weights (z_tlk = beta_lk / sum_k' beta_lk')
 * and d-hat from init_mode.  The paper gives no initial state; this is the
 * library's reading.  inputs_on_device: 1 if V, W, A, pi are device
 * pointers.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * On success *out holds the new context; on failure *out is NULL.
 */
NFHMM_API int nfhmm_vi_init(nfhmm_ctx **out, const nfhmm_dims *d,
                  const float *V, const float *W, const float *A, const float *pi,
                  int inputs_on_device, void *cuda_stream);

/*
 * nfhmm_vi_reinit -- load a new spectrogram and model of the same sizes into
 * an existing context (its device memory is reused) and reset it to the
 * initial state, as nfhmm_vi_init does.  On failure the context holds no
 * usable state: every call but another nfhmm_vi_reinit or nfhmm_destroy
 * returns NFHMM_ESTATE.  Synchronises once.
 */
NFHMM_API int nfhmm_vi_reinit(nfhmm_ctx *c, const float *V, const float *W, const float *A,
                              const float *pi, int inputs_on_device);

/*
 * nfhmm_vi_sweep -- run n_sweeps sweeps of Section 3.2.  Each sweep applies
 * Eq. 6 to the current (counts, d-hat), then recomputes counts (Eq. 7 into
 * Eq. 6's first term), phi-hat (Eq. 8) and d-hat (forward-backward per
 * source) from that alpha-hat.  bound_out: NULL, or receives the bound after
 * the last sweep (synchronises).  n_sweeps >= 0.
 */
NFHMM_API int nfhmm_vi_sweep(nfhmm_ctx *c, int n_sweeps, double *bound_out);

/*
 * nfhmm_vi_sweep_async -- queue n_sweeps >= 1 sweeps without waiting.  With
 * prepare_bound = 1 the last sweep also forms the bound's per-frame terms, so
 * that a following nfhmm_bound or nfhmm_job_bounds only reduces them.  Lets
 * a caller keep several contexts' sweeps in flight at once.
 */
NFHMM_API int nfhmm_vi_sweep_async(nfhmm_ctx *c, int n_sweeps, int prepare_bound);

/*
 * nfhmm_bound -- the variational lower bound of the current state
 * (alpha-hat of the last sweep with its optimal z-hat and d-hat), reduced in
 * FP64.  The paper prints no bound; it follows from Eq. 1 and the factorised
 * posterior of Section 3.2.  Needs at least one sweep (else NFHMM_ESTATE).
 * Synchronises.
 */
NFHMM_API int nfhmm_bound(nfhmm_ctx *c, double *out);

/*
 * nfhmm_separate -- separated spectrograms of Section 4, S x T x F.
 * masked = 0: Vhat^(s)_lt, a combination of source s's elements weighted by
 * the estimated mixture weights (weights: NFHMM_SEP_MEAN or
 * NFHMM_SEP_EXPECTATION); masked = 1: V*^(s)_lt = V_lt Vhat^(s)_lt /
 * sum_s' Vhat^(s')_lt (V/S where the denominator is 0).  Needs at least one
 * sweep.  out_on_device: 1 if out is a device pointer (then asynchronous).
 */
NFHMM_API int nfhmm_separate(nfhmm_ctx *c, float *out, int masked, int weights, int out_on_device);

/* nfhmm_get_posteriors -- d-hat (S x T x N) of the current state. */
NFHMM_API int nfhmm_get_posteriors(nfhmm_ctx *c, float *dhat, int on_device);

/* nfhmm_get_weights -- alpha-hat (T x M) of the last sweep (Eq. 6).  Needs a sweep. */
NFHMM_API int nfhmm_get_weights(nfhmm_ctx *c, float *alpha, int on_device);

/* nfhmm_get_surrogate -- phi-hat (S x T x N) of the last sweep, stored
 * without the per-frame constant -gamma*K*psi(sum_k alpha_tk) of Eq. 8
 * (it cancels in d-hat).  Needs a sweep. */
NFHMM_API int nfhmm_get_surrogate(nfhmm_ctx *c, float *phi, int on_device);

/* nfhmm_get_state / nfhmm_set_state -- checkpoint: (counts T x M,
 * d-hat S x T x N, sweeps done).  A sweep after set_state starts from Eq. 6
 * on these values; resuming from a saved state is bit-identical. */
NFHMM_API int nfhmm_get_state(nfhmm_ctx *c, float *counts, float *dhat, int *sweeps_done, int on_device);
NFHMM_API int nfhmm_set_state(nfhmm_ctx *c, const float *counts, const float *dhat, int sweeps_done,
                    int on_device);

/*
 * Batches of jobs.  A job is one spectrogram to separate; the jobs of a
 * batch share one model (W, A, pi) and sizes S, N, K, F, and each job has
 * its own number of frames.  The posterior of Section 3.2 factorises over
 * jobs (the model treats them as independent), so a batch is the sweep of
 * Section 3.2 run for every job at once: the contractions and Eqs. 6-8 over
 * all their frames together, forward-backward on one chain per (job,
 * source), and the bound as a sum of per-job bounds.  A job's results do not
 * depend on which other jobs share its batch.
 * A batch context keeps its jobs' frames back to back in a frame store of
 * d->T frames, in the order they were added; removing a job moves the later
 * jobs down.  Every call above applies to a batch context over the frames
 * of all its jobs in that order, with T the frames held (nfhmm_batch_info);
 * nfhmm_vi_init makes a batch of one job.  The sweep counter and the bound
 * of nfhmm_vi_sweep cover all jobs; a job added after a sweep starts from
 * the initial state.  Calls that need "a sweep" need one since the last
 * change of the job list.
 */

/* nfhmm_vi_init_batch -- a batch of n_jobs jobs of job_frames[j] >= 1 frames
 * (d->T = sum of job_frames); V holds their spectrograms back to back
 * (d->T x F).  job_ids: NULL or n_jobs ids, as from nfhmm_batch_add. */
NFHMM_API int nfhmm_vi_init_batch(nfhmm_ctx **out, const nfhmm_dims *d, int n_jobs,
                                  const int *job_frames, const float *V, const float *W,
                                  const float *A, const float *pi, int inputs_on_device,
                                  void *cuda_stream, long long *job_ids);

/* nfhmm_batch_create -- an empty batch with room for d->T frames and
 * max_jobs jobs, holding the model (W, A, pi; validated).  Device memory is
 * allocated here, in proportion to d->T: a batch never allocates when jobs
 * come and go. */
NFHMM_API int nfhmm_batch_create(nfhmm_ctx **out, const nfhmm_dims *d, int max_jobs,
                                 const float *W, const float *A, const float *pi,
                                 int inputs_on_device, void *cuda_stream);

/* nfhmm_batch_add -- append a job of T >= 1 frames (V: T x F), validate it
 * and set its initial state (as nfhmm_vi_init does).  *job_id receives its
 * id (unique within the context).  NFHMM_EFULL if the frames or job slots
 * left are too few; on any failure the batch is unchanged.  Synchronises. */
NFHMM_API int nfhmm_batch_add(nfhmm_ctx *c, int T, const float *V, int on_device,
                              long long *job_id);

/* nfhmm_batch_add_many -- append n jobs at once (job j: T[j] frames from
 * V[j]), validated together (one synchronisation); all or none are added.
 * job_ids: NULL or n ids. */
NFHMM_API int nfhmm_batch_add_many(nfhmm_ctx *c, int n, const int *T, const float *const *V,
                                   int on_device, long long *job_ids);

/* nfhmm_batch_remove -- drop a job and free its frames (asynchronous). */
NFHMM_API int nfhmm_batch_remove(nfhmm_ctx *c, long long job_id);

/* nfhmm_batch_remove_many -- drop n jobs and close the gaps in one pass
 * (asynchronous). */
NFHMM_API int nfhmm_batch_remove_many(nfhmm_ctx *c, int n, const long long *job_ids);

/* nfhmm_batch_info -- number of jobs, frames held, and per job (arrays of at
 * least n_jobs entries, each may be NULL): id, first frame, frames, sweeps
 * run since the job was added. */
NFHMM_API int nfhmm_batch_info(nfhmm_ctx *c, int *n_jobs, int *frames_held, long long *ids,
                               int *t0, int *T, int *sweeps);

/* nfhmm_job_bounds -- the bound of each job (in job order; they sum to
 * nfhmm_bound).  Needs a sweep.  Synchronises. */
NFHMM_API int nfhmm_job_bounds(nfhmm_ctx *c, double *bounds);

/* nfhmm_job_posteriors -- d-hat of one job, S x T_job x N. */
NFHMM_API int nfhmm_job_posteriors(nfhmm_ctx *c, long long job_id, float *dhat, int on_device);

/*
 * nfhmm_set_option -- tune a context (results change only by rounding):
 *   NFHMM_OPT_FB_CHUNK     frames per time chunk of the forward-backward (1..128)
 *   NFHMM_OPT_FB_PRODUCTS  how the chunk transfer matrices are formed:
 *                          NFHMM_FB_PRODUCTS_TC (default, and the form of
 *                          the stateless calls: split-TF32 tcgen05 MMAs over
 *                          128-row tiles) or NFHMM_FB_PRODUCTS_SIMT (FP32
 *                          FMAs on the CUDA cores, one thread per row)
 *   NFHMM_OPT_FB_GROUP     chunks per group of the two-level scan across
 *                          chunks (2..4096), 0 for a single-level scan, -1
 *                          for a size that follows the chunk length (the
 *                          default of one-job contexts; batches default to 0
 *                          and chunks of 32 frames)
 *   NFHMM_OPT_GRAPHS       1 (default): sweeps whose launch configuration
 *                          (frames, chunks, bound terms, timed by profiling
 *                          or not) has run before are replayed from captured
 *                          CUDA graphs: the run's last sweep and each profiled
 *                          sweep (events included) from one-sweep graphs, the
 *                          plain sweeps between them up to 8 to a graph;
 *                          0: launch by launch
 *   NFHMM_OPT_PROFILE_STRIDE  k >= 1 (default 1): with profiling on, the
 *                          stages of every k-th sweep of a run (the 1st,
 *                          k+1-th, ...) are bracketed by events, the others
 *                          run without them; stage launches are counted
 *                          for every sweep
 *   NFHMM_OPT_FB_MODE      0 (default): the forward-backward as a scan over
 *                          chunks (above); k >= 1: the sequential form, one
 *                          warp per (source, job, direction) running the
 *                          recursion frame by frame, k jobs' sources per
 *                          block (clamped to 4, what a block holds), on
 *                          ceil(S * jobs / k) SMs that the
 *                          contractions leave free (at most half of them).
 *                          Its latency is the longest job's frames; it suits
 *                          batches of many jobs.  The first use allocates
 *                          S x T x (N + 68) floats (NFHMM_ENOMEM if no room)
 *   NFHMM_OPT_TEST_WAIT_TIMEOUT  test hook of the failure path (tensor-core
 *                          contexts only): v in [1, 10^9] makes the next
 *                          sweep's reconstruction contraction first wait v
 *                          nanoseconds on a barrier that nothing completes.
 *                          The wait gives up as every bounded device wait
 *                          does: its block sets the error word, waits for
 *                          its own copies and tensor-core operations in
 *                          flight, frees its tensor memory and returns, and
 *                          the next call that synchronises (a bound, a host
 *                          output) returns NFHMM_ETIMEOUT.  That sweep is
 *                          launched directly, not from a captured graph, and
 *                          its state is not usable (restore one with
 *                          nfhmm_set_state); the context stays usable.
 *                          0 clears a pending hook
 *   NFHMM_OPT_TILE_GEMM1   column tile of the reconstruction contraction
 *                          (Vhat = beta w, output columns = frequencies) on
 *                          the tensor cores: 64, 96 or 128 (FP32; default
 *                          128), or 64, 96, 128 or 192 (BF16)
 *   NFHMM_OPT_TILE_GEMM2   column tile of the back-projection (counts,
 *                          output columns = elements): 64, 96, 128 or 160
 *                          (FP32; default 160), or also 192 (BF16)
 *   NFHMM_OPT_TILE_STAGES1, NFHMM_OPT_TILE_STAGES2  depth of each
 *                          contraction's shared-memory ring of operand
 *                          stages: 0 (default) the deepest that fits the
 *                          tile, else 2 .. that depth (NFHMM_Q_TILE_STAGES*
 *                          reads it back).  A new column tile that cannot
 *                          hold the depth falls back to 0; a depth asked for
 *                          beyond the tile's deepest is rejected
 *   NFHMM_OPT_TILE_EPI_STAGE1, NFHMM_OPT_TILE_EPI_STAGE2  1: the epilogue's
 *                          second operand (V for the reconstruction, w for the
 *                          back-projection) is copied into shared memory for
 *                          each tile while its MMAs run, instead of being
 *                          read from global memory 16 columns at a time after
 *                          them; it takes ring depth (some FP32 tiles cannot
 *                          hold it: NFHMM_EINVAL).  0 (default): not staged
 *   NFHMM_OPT_TILE_PREFETCH1, NFHMM_OPT_TILE_PREFETCH2  L2 prefetch distance
 *                          of each contraction's operand copies: 0 (default)
 *                          none, else 1..64 K-blocks beyond the ring are
 *                          asked into L2 ahead of their copies
 *                          Every row tile is 128 frames; results differ
 *                          between tile shapes only by rounding (the order
 *                          of the accumulation and of the bound's partial
 *                          sums).  Tensor-core contexts only (NFHMM_EINVAL
 *                          otherwise); synchronises.
 */
#define NFHMM_OPT_FB_CHUNK    0
#define NFHMM_OPT_FB_PRODUCTS 1
#define NFHMM_OPT_GRAPHS      2
#define NFHMM_OPT_FB_GROUP    3
#define NFHMM_OPT_PROFILE_STRIDE 4
#define NFHMM_OPT_FB_MODE     5
#define NFHMM_OPT_TEST_WAIT_TIMEOUT 6
#define NFHMM_OPT_TILE_GEMM1  7
#define NFHMM_OPT_TILE_GEMM2  8
#define NFHMM_OPT_TILE_STAGES1 9
#define NFHMM_OPT_TILE_STAGES2 10
#define NFHMM_OPT_TILE_PREFETCH1 11
#define NFHMM_OPT_TILE_PREFETCH2 12
#define NFHMM_OPT_TILE_EPI_STAGE1 13
#define NFHMM_OPT_TILE_EPI_STAGE2 14

/*
 * nfhmm_autotune -- choose the forward-backward form and geometry, then the
 * contractions' tile shapes, for the context's current jobs by timing whole
 * sweeps on them.  Forward-backward first: the scan with every
 * candidate chunk length in {8, 12, 16, 20, 24, 32, 48, 64} (at most the
 * longest job's frames), with groups of the automatic size and without
 * groups, then the sequential form (NFHMM_OPT_FB_MODE) with 1, 2 and 4 jobs'
 * sources per block (as far as a block holds them).  Then, with the form
 * chosen and on tensor-core contexts, the tile shapes one coordinate at a
 * time: the reconstruction's column tile over NFHMM_OPT_TILE_GEMM1's
 * choices, the back-projection's over NFHMM_OPT_TILE_GEMM2's, the staging
 * of each epilogue operand, then each ring depth from 2 to the deepest, then
 * each L2 prefetch distance over
 * {0, 4, 8, 16} (read back with NFHMM_Q_TILE_*).  Each
 * candidate runs two
 * sweeps (which capture its graph) and then `reps` sweeps (reps <= 0: 3)
 * between CUDA events, every trial starting from the same state: the counts,
 * posteriors, alpha-hat and log normalisers are copied aside first and put
 * back at the end, so the
 * context's posteriors, bound and flags are unchanged (the bound of the current
 * state is formed before the trials if it was not yet); it needs room for that
 * copy (NFHMM_ENOMEM otherwise).  The fastest candidate is then set as by
 * NFHMM_OPT_FB_CHUNK, NFHMM_OPT_FB_GROUP and NFHMM_OPT_FB_MODE.  Needs a sweep over the current
 * jobs (NFHMM_ESTATE otherwise).  Writes the chosen chunk length, group size
 * and its mean sweep time in microseconds to the non-NULL outputs; the chosen
 * form is read back with NFHMM_Q_FB_MODE.
 * Synchronises.
 */
NFHMM_API int nfhmm_autotune(nfhmm_ctx *c, int reps, int *chunk_out, int *group_out,
                             double *us_out);
#define NFHMM_FB_PRODUCTS_SIMT 0
#define NFHMM_FB_PRODUCTS_TC   1
NFHMM_API int nfhmm_set_option(nfhmm_ctx *c, int key, long long value);

/*
 * nfhmm_serve -- continuous batching of separation requests over batch
 * contexts (one per model; created empty with nfhmm_batch_create).  Each
 * request runs sweeps until its own bound changes by less than
 * rel_tol * |bound| between two sweeps (after at least min_sweeps), or
 * max_sweeps; it then leaves with its posteriors.  A request is admitted to
 * its model's batch, in arrival order, once it has arrived and the batch has
 * room for its frames (else it waits; a request larger than an empty batch
 * fails with NFHMM_EFULL).  Every tick runs one sweep of each non-empty
 * batch.  Times are seconds from the start of the call.  With realtime = 1 a
 * request arrives at arrival_s on the host clock; with 0 all have arrived at
 * the start.  Synchronises; returns when every request is done.  The paper
 * has no serving loop: convergence by relative bound change is the
 * library's reading of "until convergence".
 */
typedef struct {
  int model;          /* index of the batch context that serves it          */
  int T;              /* frames (>= 1)                                      */
  const float *V;     /* T x F, host memory                                 */
  double arrival_s;   /* arrival time                                        */
  float *dhat_out;    /* NULL, or S x T x N host buffer for the posteriors  */
} nfhmm_request;
typedef struct {
  double rel_tol;     /* convergence tolerance on the bound (e.g. 1e-5)     */
  int min_sweeps;     /* >= 1                                               */
  int max_sweeps;     /* >= min_sweeps                                      */
  int realtime;       /* 1: honour arrival_s; 0: everything queued at start */
} nfhmm_serve_opts;
typedef struct {
  double admit_s;     /* time the request joined its batch (-1 if never)   */
  double done_s;      /* time its posteriors were out                       */
  int sweeps;         /* sweeps it ran                                      */
  double bound;       /* its bound after the last sweep                     */
  int status;         /* NFHMM_OK or the error that ended it                */
} nfhmm_result;
NFHMM_API int nfhmm_serve(nfhmm_ctx **batches, int n_batches, const nfhmm_request *reqs,
                          int n_reqs, const nfhmm_serve_opts *opts, nfhmm_result *results);

/*
 * Exact inference in the original N-FHMM -- the comparison system of
 * Section 5, whose model opens Section 2.2: each frame t and joint state
 * c = (d^(1), ..., d^(S)) has its own maximum-likelihood mixture weights
 * theta_t(c) over the S*K elements that c selects (element index
 * (s*N + d^(s))*K + j).  One EM iteration: the frame log-likelihoods
 * l_t(c) = sum_f V_tf log sum_k theta_t(c)_k beta_k(f) for all N^S joint
 * states, forward-backward over the joint chain (transitions prod_s A^(s),
 * initial prod_s pi^(s)) for the posteriors gamma_t(c) and log P(V | theta),
 * then theta_t(c)_k <- theta_t(c)_k sum_f beta_k(f) V_tf / Vhat_tc(f),
 * normalised.  Weights start uniform.  Its cost grows as N^S: it is the
 * yardstick of the paper's per-iteration comparison, not a separation path.
 * Same V, W, A, pi layouts as nfhmm_vi_init; d->precision NFHMM_FP32 or
 * NFHMM_BF16 (the contractions); gamma and init_mode are not used.
 * Limits: S*K <= 64, N^S <= 4096.  Joint states are numbered with the last
 * source's state varying fastest.
 */
typedef struct nfhmm_exact nfhmm_exact;
NFHMM_API int nfhmm_exact_create(nfhmm_exact **out, const nfhmm_dims *d, const float *V,
                                 const float *W, const float *A, const float *pi,
                                 int inputs_on_device, void *cuda_stream);
/* n_iter >= 1 EM iterations; loglik_out: NULL, or log P(V | theta) of the
 * weights the last iteration started from (synchronises). */
NFHMM_API int nfhmm_exact_iterate(nfhmm_exact *x, int n_iter, double *loglik_out);
/* gamma: T x N^S posteriors of the last iteration's E-step. */
NFHMM_API int nfhmm_exact_posteriors(nfhmm_exact *x, float *gamma, int on_device);
/* theta: T x N^S x (S*K) current weights. */
NFHMM_API int nfhmm_exact_weights(nfhmm_exact *x, float *theta, int on_device);
NFHMM_API void nfhmm_exact_destroy(nfhmm_exact *x);

/* nfhmm_destroy -- free the context and its device memory (waits for its work). */
NFHMM_API void nfhmm_destroy(nfhmm_ctx *c);

/* nfhmm_last_error -- message of the calling thread's last failure ("" if none). */
NFHMM_API const char *nfhmm_last_error(void);

/*
 * nfhmm_forward_backward -- stateless forward-backward for S independent
 * chains (the q(D^(s)) step of Section 3.2), all pointers on device:
 * phi S x T x N (emissions exp(phi)), A S x N x N row-stochastic, pi S x N;
 * writes dhat S x T x N and logZ[S] (FP64 log normalisers).  chunk_len: frames
 * per time chunk of the parallel-in-time form (0 = library default; values
 * above 128 are clamped to 128 and values above T to T, so T > 128 always
 * gives ceil(T / L) chunks).  Allocates its scratch on the stream.
 * Asynchronous.  A failure on the device has no context to report it
 * through: if a bounded device wait gave up, or a chain's normaliser
 * vanished (data of probability zero under the chain: a transition or an
 * emission that excludes every state), every logZ[s] is set to NaN and d-hat
 * is undefined; check logZ once the stream has been synchronised.
 */
NFHMM_API int nfhmm_forward_backward(int S, int N, int T, const float *phi, const float *A,
                           const float *pi, float *dhat, double *logZ, int chunk_len,
                           void *cuda_stream);

/*
 * nfhmm_forward_backward_noalloc -- the same computation, arguments and
 * results as nfhmm_forward_backward, for callers that must not allocate
 * device memory when they call in: processes whose device memory belongs to
 * another allocator (a serving runtime with a fixed HBM budget, a host
 * framework that owns every byte) or latency-critical threads that cannot
 * risk cudaMalloc/cudaFree, which may block and synchronise the device.  The
 * paper has no counterpart; this is a property of the interface only.
 * The call allocates nothing: its scratch is one fixed device array of
 * NFHMM_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits.  A problem needs about
 * 8*S*(C + C')*(P*P + N) + 12*S*(C + C') bytes, C = ceil(T/L) chunks of L frames
 * (L at most 128; by default 0.3*sqrt(T) rounded, clamped to [8, 64]), C' =
 * ceil(C/G) groups of G = ceil(sqrt(C/2)) chunks (none below 24 chunks),
 * P = 8*ceil(N/8), plus, when there are groups, 256*S*C*ceil(P/32)*P16 bytes
 * of tensor-core operand images (P16 = P rounded up to a multiple of 16), plus
 * alignment; larger problems are rejected with NFHMM_EINVAL and a message
 * giving both sizes.
 * The first call on a device looks up the array's device address (with that
 * device current) and should be made before any stream capture.  All calls
 * share the array and it keeps the last call's contents: calls whose work
 * overlaps on the GPU (different streams, or different host threads without
 * ordering) race on it.  Asynchronous; inputs and outputs on the device.
 * Device-side failures are reported as by nfhmm_forward_backward: every
 * logZ[s] NaN.
 */
#define NFHMM_NOALLOC_SCRATCH_BYTES (32u << 20)
NFHMM_API int nfhmm_forward_backward_noalloc(int S, int N, int T, const float *phi,
                                             const float *A, const float *pi, float *dhat,
                                             double *logZ, int chunk_len, void *cuda_stream);

/*
 * nfhmm_mma_rate -- the measured dense rate (TFLOP/s, FP32 accumulate) of
 * this GPU's tcgen05 tensor cores for the operand kind of a precision:
 * NFHMM_FP32 times kind::tf32 MMAs (one pass; the split-TF32 contractions
 * issue three per product, so their ceiling is a third of it), NFHMM_BF16
 * kind::f16 MMAs on bf16 operands.  Every SM issues back-to-back 128 x 256
 * MMAs (K = 8 tf32 or 16 bf16 per instruction) from shared memory into one
 * TMEM accumulator; the launches are timed with CUDA events on cuda_stream.
 * The paper has no counterpart: this is the denominator of the contractions'
 * roofline.  Allocates 4 bytes of device memory; synchronises.
 */
NFHMM_API int nfhmm_mma_rate(int precision, double *tflops_out, void *cuda_stream);

/*
 * nfhmm_digamma -- the library's device psi and exp(psi) on n values x >= 1
 * (device pointers; psi_out or w_out may be NULL).  Asynchronous.
 */
NFHMM_API int nfhmm_digamma(const float *x, float *psi_out, float *w_out, size_t n, void *cuda_stream);

/*
 * Profiling: with profiling on, every kernel stage a context runs (of every
 * k-th sweep, NFHMM_OPT_PROFILE_STRIDE) is
 * bracketed by CUDA events on the stream it runs on.  nfhmm_profile_read
 * synchronises and returns, for one stage since the last reset, the summed
 * event time (ms), the number of stage invocations and of kernel launches.
 */
#define NFHMM_STAGE_WEIGHTS 0  /* Eq. 6, psi, Eq. 8                        */
#define NFHMM_STAGE_GEMM1   1  /* reconstruction Vhat and ratio V/Vhat     */
#define NFHMM_STAGE_GEMM2   2  /* back-projection and counts (Eq. 7 -> 6)  */
#define NFHMM_STAGE_FB      3  /* forward-backward, all phases             */
#define NFHMM_STAGE_BOUND   4  /* bound reduction                          */
#define NFHMM_STAGE_INIT    5  /* inputs, validation and initial state     */
#define NFHMM_NUM_STAGES    6
NFHMM_API int nfhmm_profile_enable(nfhmm_ctx *c, int on);
NFHMM_API int nfhmm_profile_read(nfhmm_ctx *c, int stage, double *ms_total,
                                 long long *invocations, long long *launches, int reset);

/* nfhmm_kernel_launches -- number of kernels this context has launched. */
NFHMM_API long long nfhmm_kernel_launches(nfhmm_ctx *c);

/*
 * nfhmm_query -- read one property of a context into *value:
 *   NFHMM_Q_TENSOR_CORES  1 if the contractions run on tcgen05 tensor cores
 *   NFHMM_Q_FB_CHUNK      frames per time chunk of the forward-backward
 *   NFHMM_Q_SWEEPS_DONE   sweeps run since the initial state
 *   NFHMM_Q_DEVICE_BYTES  device memory the context holds
 *   NFHMM_Q_FRAME_CAPACITY, NFHMM_Q_MAX_JOBS  the batch's room
 */
#define NFHMM_Q_TENSOR_CORES 0
#define NFHMM_Q_FB_CHUNK     1
#define NFHMM_Q_SWEEPS_DONE  2
#define NFHMM_Q_DEVICE_BYTES 3
#define NFHMM_Q_FRAME_CAPACITY 4   /* frames the context's frame store holds */
#define NFHMM_Q_MAX_JOBS       5   /* jobs the context can hold            */
#define NFHMM_Q_FB_GROUP       6   /* chunks per group of the scan (0: none) */
#define NFHMM_Q_FB_MODE        7   /* 0: scan; k >= 1: sequential, k per block */
#define NFHMM_Q_TILE_GEMM1     8   /* column tile of the reconstruction (0: not tensor cores) */
#define NFHMM_Q_TILE_GEMM2     9   /* column tile of the back-projection   */
#define NFHMM_Q_TILE_STAGES1  10   /* ring depth of the reconstruction     */
#define NFHMM_Q_TILE_STAGES2  11   /* ring depth of the back-projection    */
#define NFHMM_Q_TILE_PREFETCH1 12  /* L2 prefetch distance, reconstruction */
#define NFHMM_Q_TILE_PREFETCH2 13  /* L2 prefetch distance, back-projection */
#define NFHMM_Q_TILE_EPI_STAGE1 14 /* epilogue operand staged, reconstruction */
#define NFHMM_Q_TILE_EPI_STAGE2 15 /* epilogue operand staged, back-projection */
NFHMM_API int nfhmm_query(nfhmm_ctx *c, int key, long long *value);

#ifdef __cplusplus
}
#endif

#endif /* NFHMM_H */
