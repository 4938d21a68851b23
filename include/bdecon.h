/*
 * bdecon.h -- C ABI of libbdecon: GB300 (sm_103a) posterior sampling for
 * Bayesian deconvolution of microscopy frames (Hendrix et al., "Re-thinking
 * Richardson-Lucy without Iteration Cutoffs: Physically Motivated Bayesian
 * Deconvolution", arXiv 2411.00991).
 *
 * The library samples the posterior of Eq. 9 over a strictly positive
 * object rho on the camera grid padded by the PSF radius R (Fig. 5b):
 *   likelihood  Eq. 1-6: mu = PSF (x) rho integrated over each pixel, photon
 *               counts Poisson(mu_n) summed out against the sCMOS readout
 *               Normal(G_n phi + o_n, var_n);
 *   prior       Eq. 7-8: Dirichlet on |F(rho)| / sum|F(rho)| with
 *               hyperparameter |OTF| / sum|OTF|, taken per stride x stride
 *               patch aligned with the sub-lattice (the paper's locality
 *               argument, Methods "Parallelization Technique");
 *   sampler     one Metropolis-Hastings step per object pixel per sweep
 *               (the pixel-wise Gibbs scan of Fig. 5d), pixels of one
 *               sub-lattice class (i mod S, j mod S) updated in parallel,
 *               classes in raster order; log-space Gaussian random-walk
 *               proposals from Philox4x32-10 keyed by (seed) with counter
 *               (pixel, sweep, chain, 0).
 * The estimator is the mean of the post-burn-in samples (Results; Methods
 * after Eq. 9).
 *
 * Conventions for every entry point:
 *   - Every call returns a bdecon_status; nothing aborts the process.
 *     bdecon_last_error(handle) returns a message for the last failure on
 *     that handle (for handle-less failures pass NULL: thread-local).
 *   - "host" pointers are ordinary CPU memory, read or written before the
 *     call returns.  Work is queued on the CUDA stream given at creation;
 *     calls that return data to the host synchronise that stream first.
 *   - Images are row-major, row index first.  Object arrays are
 *     (H + 2R) x (W + 2R) with R = (L - 1) / 2.
 *   - The handle owns all device memory it allocates (or borrows the
 *     caller's workspace, see bdecon_create_in); bdecon_destroy frees it.
 *   - Device-side failures (a sub-lattice wait that timed out, a
 *     non-finite expected image) set a flag that the next bdecon_sync (or
 *     any call that reads results) returns as BDECON_ERR_TIMEOUT or
 *     BDECON_ERR_NUMERIC; the handle then refuses further sweeps.
 */
#ifndef BDECON_H
#define BDECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bdecon_handle bdecon_handle;

typedef enum {
    BDECON_OK = 0,
    BDECON_ERR_INVALID = 1,   /* bad argument; nothing was changed          */
    BDECON_ERR_NOMEM = 2,     /* device memory (or caller workspace) short  */
    BDECON_ERR_CUDA = 3,      /* a CUDA runtime call failed                 */
    BDECON_ERR_TIMEOUT = 4,   /* a bounded device-side wait gave up         */
    BDECON_ERR_STATE = 5,     /* call not allowed in the handle's state     */
    BDECON_ERR_NUMERIC = 6    /* non-finite value met on the device         */
} bdecon_status;

typedef enum {
    BDECON_FP64 = 0,          /* plain sampler, all arithmetic in double    */
    BDECON_FP32 = 1           /* float sweeps; double refresh and trace     */
} bdecon_precision;

/* One deconvolution problem (a camera frame and its calibration).  All
 * pointers are host pointers, copied by the create call.                   */
typedef struct {
    int32_t H, W;              /* frame size, >= 1                                  */
    const float* image;        /* H*W readout w_n in ADU (Eq. 4)                    */
    int32_t L;                 /* PSF side, odd, 1 <= L <= 63                       */
    const double* psf;         /* L*L pixel-integrated PSF, >= 0, sum > 0; the
                                  library normalises it to sum 1 (Eq. 1-2)          */
    const float* gain_map;     /* H*W gain G_n (ADU/photon) or NULL -> gain         */
    double gain;
    const float* offset_map;   /* H*W offset o_n (ADU) or NULL -> offset            */
    double offset;
    const float* var_map;      /* H*W read-noise variance (ADU^2) or NULL -> read_var */
    double read_var;
    int32_t stride;            /* sub-lattice stride = prior patch side S; 0 -> L
                                  (L + f - 1 with subpixel f); must be >= that.  Part
                                  of the model (it sets the prior's patches).       */
    int32_t n_chains;          /* independent chains, >= 1                          */
    uint64_t seed;             /* Philox key                                        */
    double step;               /* sd of the log-space random walk; 0 -> 0.2         */
    int32_t burn_in;           /* sweeps t <= burn_in are not averaged              */
    int32_t refresh_every;     /* recompute mu, spectra and log posterior from rho
                                  in double every this many sweeps (0 -> never
                                  after creation)                                   */
    int32_t precision;         /* bdecon_precision                                  */
    int32_t max_sweeps;        /* capacity of the per-sweep trace; 0 -> 4096        */
    int32_t flags;             /* BDECON_FLAG_*                                     */
    int32_t team_warps;        /* warps cooperating on one pixel update, 1..8; 0 ->
                                  automatic from the problem alone (1 warp when
                                  n_chains x patches >= 2048, else one warp per 100
                                  PSF-window pixels).  It fixes the order of the
                                  per-update float reductions, so a problem gives
                                  the same chain alone or in any batch and plan.  */
    int32_t sample_every;      /* keep the object after every this-many-th sweep past
                                  burn_in (0 -> 1): the candidate images from which
                                  quantiles and credible intervals are taken        */
    int32_t n_samples;         /* kept objects per chain, >= 0 (0: none kept); the
                                  sweep t > burn_in with (t - burn_in) a multiple of
                                  sample_every goes to slot (t - burn_in) /
                                  sample_every - 1 while that is < n_samples        */
    double adapt_target;       /* 0: every pixel proposes with `step`.  In (0, 1):
                                  during burn-in each pixel m adapts its own scale
                                  s_m (from `step`): after its update in sweep t,
                                  s_m *= exp(g (1 - adapt_target)) if accepted,
                                  exp(-g adapt_target) if not, g = 0.5/sqrt(t),
                                  clamped to [1e-4, 4]; fixed after burn-in      */
    int32_t subpixel;          /* object lattice cells per camera pixel side f, 0..8
                                  (0 -> 1: the camera grid).  With f > 1 the object
                                  lives on a lattice f times finer (the paper's
                                  Nyquist lattice); psf is given on that lattice and
                                  each camera pixel sums its f x f cells (Eq. 1):
                                  mu[a][b] = sum Ke[p][q] rho[f a+Le-1-p][f b+Le-1-q],
                                  Ke = psf (x) box_f of side Le = L + f - 1.  The
                                  object is (f H + L - 1) x (f W + L - 1); stride
                                  defaults to Le and must be >= Le.                */
} bdecon_problem;

#define BDECON_FLAG_ACCEPT_LOG 1   /* keep the accept decision of every update of
                                      every sweep (max_sweeps x object bytes; testing) */
#define BDECON_FLAG_SECOND_MOMENT 2 /* also accumulate sum of rho^2 (uncertainty)  */
#define BDECON_FLAG_AUGMENTED 4    /* photon-count augmented sampler: each sweep first
                                      draws every camera pixel's photon count phi_n from
                                      p(phi | w_n, mu_n) (the completed likelihood of
                                      Eq. 5), then updates rho against the Poisson
                                      likelihood sum_n phi_n log mu_n - mu_n; the rho-
                                      marginal of its target is Eq. 9.  Its trace is the
                                      log of the joint density p(w, phi, rho).      */

/* ------------------------------------------------------------- lifetime */

/* Bytes of device workspace bdecon_create_in needs for these problems.     */
bdecon_status bdecon_workspace_size(const bdecon_problem* problems, int32_t n_problems,
                                    size_t* bytes);

/* Create a sampler over one problem.  Validates the inputs, copies them to
 * the device (host -> device), normalises the PSF, derives the Dirichlet
 * hyperparameters and per-pixel constants, draws the initial object
 * (rho0_m = b0 exp(z_m / 10) with b0 = max(0.1, mean_n (w_n - o_n)/G_n) and
 * z_m the Philox normal of counter (m, 0, chain, 0)) and runs the double-
 * precision refresh (Eq. 1-2, 8, 9).  stream: a cudaStream_t or NULL.
 * On failure *out is NULL and nothing stays allocated.                     */
bdecon_status bdecon_create(const bdecon_problem* problem, void* stream, bdecon_handle** out);

/* Same for a batch of problems of any sizes, PSFs and chain counts (one
 * precision).  By default the problems are grouped by PSF side, stride and
 * update team, and each group's chains run in one persistent cooperative
 * launch of the sweep kernel per segment of sweeps (bdecon_set_grouping(h, 1)
 * puts every problem in one launch; bdecon_autotune picks the faster).  A
 * problem's results do not depend on the rest of the batch.               */
bdecon_status bdecon_batch_create(const bdecon_problem* problems, int32_t n_problems,
                                  void* stream, bdecon_handle** out);

/* As bdecon_batch_create, placing all device state in the caller's device
 * buffer (at least bdecon_workspace_size bytes, 256-byte aligned).  The
 * caller keeps ownership and must keep it alive until bdecon_destroy.      */
bdecon_status bdecon_create_in(const bdecon_problem* problems, int32_t n_problems, void* stream,
                               void* device_workspace, size_t bytes, bdecon_handle** out);

void bdecon_destroy(bdecon_handle* h);

const char* bdecon_last_error(const bdecon_handle* h);

/* --------------------------------------------------------------- sampling */

/* Queue n sweeps of every chain (asynchronous on the handle's stream): the
 * paper's pixel-by-pixel sampler, each pixel drawn from its conditional
 * given the rest of the object, with the pixels that are conditionally
 * independent (windows beyond the PSF support) updated in parallel (Methods,
 * "Parallelization Technique"; Fig. 5c-d).  Here each pixel update is one
 * Metropolis-Hastings step with a log-space random walk.  A sweep visits the
 * S*S sub-lattice classes in raster order of the in-patch offset (u, v);
 * every pixel of a class is updated once.  After sweep t the
 * object is added to the running sum when t > burn_in, and mu, the patch
 * spectra and the log posterior are recomputed in double when t is a
 * multiple of refresh_every.  Errors: BDECON_ERR_STATE after a device
 * failure, BDECON_ERR_INVALID if the trace capacity would be exceeded.     */
bdecon_status bdecon_sweep(bdecon_handle* h, int32_t n);

/* Wait for queued work; returns the device error flag, if any.             */
bdecon_status bdecon_sync(bdecon_handle* h);

/* ---------------------------------------------------------------- results */

/* Posterior mean of problem p over all its chains and all sweeps t >
 * burn_in so far -- the paper's estimate of the object, the average of the
 * sampled objects after burn-in (Results; the text after Eq. 9) -- in
 * double, into host out: (H+2R)*(W+2R) values, or the H*W central crop when
 * crop != 0.  BDECON_ERR_STATE if no sweep has been
 * averaged yet.                                                            */
bdecon_status bdecon_posterior_mean(bdecon_handle* h, int32_t p, double* out, int32_t crop);

/* Per-pixel posterior variance (needs BDECON_FLAG_SECOND_MOMENT), same
 * layout and pooling as bdecon_posterior_mean.                             */
bdecon_status bdecon_posterior_var(bdecon_handle* h, int32_t p, double* out, int32_t crop);

/* Uncertainty maps pooled over the chains of problem p, laid out as
 * bdecon_posterior_mean (both need BDECON_FLAG_SECOND_MOMENT): the posterior
 * standard deviation sqrt(var), and the coefficient of variation std / mean
 * (the paper's relative uncertainty map).                                  */
bdecon_status bdecon_posterior_std(bdecon_handle* h, int32_t p, double* out, int32_t crop);
bdecon_status bdecon_posterior_cv(bdecon_handle* h, int32_t p, double* out, int32_t crop);

/* Photon counts phi_n of chain c of an augmented problem (H*W doubles):
 * those of the last sweep (or of the initial draw).                        */
bdecon_status bdecon_get_phi(bdecon_handle* h, int32_t p, int32_t c, double* out);

/* Per-pixel proposal scales of chain c of problem p, (H+2R)*(W+2R)
 * doubles: the adapted s_m (see adapt_target), else `step` everywhere.   */
bdecon_status bdecon_get_steps(bdecon_handle* h, int32_t p, int32_t c, double* out);

/* The kept objects of chain c of problem p (see n_samples), oldest first,
 * each (H+2R)*(W+2R) doubles, into host out (capacity cap doubles); *n
 * receives the doubles available (kept objects x object pixels).          */
bdecon_status bdecon_get_samples(bdecon_handle* h, int32_t p, int32_t c, double* out, size_t cap,
                                 size_t* n);

/* Per-pixel quantiles of the kept objects of all chains of problem p, for
 * each of nq (1..64) probabilities q[k] in [0, 1]: with the n kept values of
 * a pixel sorted, x_(0) <= ... <= x_(n-1), the value at h = (n - 1) q is
 * x_(floor h) + (h - floor h)(x_(floor h + 1) - x_(floor h)) (linear
 * interpolation between order statistics).  out: nq maps, each laid out as
 * bdecon_posterior_mean.  Sorting runs on the device; at most 8192 kept
 * values per pixel (kept objects x chains).                                */
bdecon_status bdecon_posterior_quantiles(bdecon_handle* h, int32_t p, const double* q, int32_t nq,
                                         double* out, int32_t crop);

/* Log posterior (Eq. 9 without the constant log B(alpha) terms) of chain c
 * of problem p after each sweep so far, into host out (capacity cap);
 * *n receives the number of sweeps.  Between refreshes the value is the
 * double running sum of the accepted changes (dL + dP); at each refresh it
 * is the double evaluation of the state.                                   */
bdecon_status bdecon_log_posterior_trace(bdecon_handle* h, int32_t p, int32_t c, double* out,
                                         size_t cap, size_t* n);

/* Accepted updates of chain c of problem p in each sweep so far.           */
bdecon_status bdecon_accept_counts(bdecon_handle* h, int32_t p, int32_t c, int64_t* out,
                                   size_t cap, size_t* n);

/* Accept decisions (1/0) of every update of chain c of problem p in every
 * sweep so far, [sweep][object pixel]; needs BDECON_FLAG_ACCEPT_LOG.  cap is
 * in bytes; *n receives sweeps * (H+2R) * (W+2R).                          */
bdecon_status bdecon_accept_log(bdecon_handle* h, int32_t p, int32_t c, uint8_t* out, size_t cap,
                                size_t* n);

/* Current object of chain c (host double, (H+2R)*(W+2R)) and the number of
 * sweeps done.                                                              */
bdecon_status bdecon_get_state(bdecon_handle* h, int32_t p, int32_t c, double* rho,
                               int64_t* sweeps);

/* Replace the object of chain c (all values > 0 and finite) and its sweep
 * counter, then refresh mu, spectra and log posterior in double.  The
 * running sums are cleared.  This is exact resume from a checkpoint: the
 * random numbers depend only on (seed, pixel, sweep, chain).               */
bdecon_status bdecon_set_state(bdecon_handle* h, int32_t p, int32_t c, const double* rho,
                               int64_t sweeps);

/* Current incrementally maintained expected image mu of chain c (H*W).      */
bdecon_status bdecon_get_mu(bdecon_handle* h, int32_t p, int32_t c, double* mu);

/* Double evaluation of Eq. 9 at the current object of chain c, without
 * changing any state.                                                       */
bdecon_status bdecon_log_posterior(bdecon_handle* h, int32_t p, int32_t c, double* out);

/* The sweep kernel's own arithmetic (in the handle's precision) for one
 * hypothetical update of object pixel m of chain c to rho_new, at the
 * current state: likelihood change dL (Eq. 6 over the PSF window), prior
 * change dP (Eq. 8 for the pixel's patch) and whether the proposal is
 * possible (all new mu > 0 and no new spectrum coefficient exactly 0).     */
bdecon_status bdecon_delta(bdecon_handle* h, int32_t p, int32_t c, int64_t m, double rho_new,
                           double* dL, double* dP, int32_t* ok);

/* ------------------------------------------------------------- scheduling */

/* Override the launch plan of problem p: tile = tile_i x tile_j patches
 * per thread block (0 for either: automatic tiles), warps per block of the
 * problem's launch group (1..8, at least the update team's; 0: the team's
 * own).  Any plan gives bit-identical results (each update's arithmetic and
 * reduction order are fixed by L alone); a plan whose blocks cannot all be
 * resident is refused with BDECON_ERR_INVALID and the previous plan kept.   */
bdecon_status bdecon_set_plan(bdecon_handle* h, int32_t p, int32_t tile_i, int32_t tile_j,
                              int32_t warps);

/* Launch plan in use: blocks of the sweep kernel, warps per block, tile
 * shape of problem p.                                                       */
/* CUDA-graph mode (enable = 1): each bdecon_sweep call runs as one graph
 * launch; its kernels (per segment: reset, the sweep launches, trace, double
 * refreshes) are captured on first use for that segment sequence and
 * replayed after (up to 8 sequences cached; a new plan or fault setting
 * drops them).  Results are identical to plain launches.  With timing on,
 * bdecon_sweep_kernel_time then reports whole-graph durations.  enable = 0
 * returns to plain launches.                                               */
bdecon_status bdecon_set_graph(bdecon_handle* h, int32_t enable);

/* Launch grouping: 0 (default) = one cooperative launch per group of
 * problems sharing PSF side, stride and update team; 1 = one launch over
 * every problem (block size the largest team, shared memory the largest
 * tile plan).  Resets warps set by bdecon_set_plan.  Results do not change. */
bdecon_status bdecon_set_grouping(bdecon_handle* h, int32_t one_launch);

/* Autotuner: times trial segments of trial_sweeps sweeps (1..64) for each
 * launch shape -- per-group launches with 1x/2x/4x the team's warps, tile
 * state resident in shared memory or streamed from global, each group tuned
 * on its own; and the same shapes as one launch over every problem -- keeps
 * the fastest, and restores the chains exactly (a device copy of the whole
 * workspace is taken first: BDECON_ERR_NOMEM if it does not fit).  Tiles
 * become automatic.  Outputs (optional): the grouping chosen and the
 * measured device milliseconds per sweep.  Synchronous.                   */
bdecon_status bdecon_autotune(bdecon_handle* h, int32_t trial_sweeps, int32_t* one_launch,
                              double* ms_per_sweep);

/* Tuning cache (process-wide; no counterpart in the paper, which describes
 * no implementation).  Each successful bdecon_autotune stores its choices
 * (grouping; per group: warps per block, resident or streamed tile state,
 * window staging) keyed by the device, the precision, the handle's staging
 * setting and every problem's frame size, PSF side, stride, lattice factor,
 * chain count, sampler and update team, in order.  A handle created later
 * for the same key (bdecon_create, _batch_create, _create_in) starts with
 * that plan instead of the automatic one; tiles are planned as usual.  A
 * plan never changes a chain's results, only its speed.  enable 0 clears the
 * cache and turns it off, 1 clears it and turns it on (the default).
 * Thread-safe.                                                              */
bdecon_status bdecon_set_tuning_cache(int32_t enable);

bdecon_status bdecon_get_plan(bdecon_handle* h, int32_t p, int32_t* blocks, int32_t* warps,
                              int32_t* tile_i, int32_t* tile_j);

/* Window staging (float problems of the marginal sampler on the camera
 * grid, PSF side <= 61): with enable = 1, plans other than the one-patch
 * one-team form copy each update's expected-image and cumulant window -- the
 * data the per-pixel update reads over the PSF window (Methods, Eq. 6;
 * Fig. 5d) -- and, when tile state is streamed, its patch spectrum (Eq. 8)
 * into shared memory with the TMA engine, the next update's copy in flight
 * while the current one computes.  Its buffers lower the blocks per SM, so
 * it is off by default and bdecon_autotune tries it.  Results do not change.
 * bdecon_get_staging reports whether problem p's launch group is staged.   */
bdecon_status bdecon_set_staging(bdecon_handle* h, int32_t enable);
bdecon_status bdecon_get_staging(bdecon_handle* h, int32_t p, int32_t* staged);

/* Lean kernel form (float problems of the marginal sampler on the camera
 * grid, unstaged plans other than the one-patch one-team form): each update
 * thread holds half as many window cells in flight (the window of Eq. 6 over
 * the PSF support, Fig. 5d) and the kernel is built for 64 registers a
 * thread, so more blocks are resident per SM.  mode -1 (the default): used
 * for PSF windows of more than 256 pixels (side 17 and up; measured faster
 * there, slower for smaller windows); 0: never; 1: wherever eligible.
 * bdecon_autotune tries both.  Results do not change.
 * bdecon_get_lean reports whether problem p's launch group runs it.        */
bdecon_status bdecon_set_lean(bdecon_handle* h, int32_t mode);
bdecon_status bdecon_get_lean(bdecon_handle* h, int32_t p, int32_t* lean);

/* Kernel launches issued by this handle since creation.                    */
bdecon_status bdecon_launch_count(const bdecon_handle* h, int64_t* launches);

/* Failure-detection test knob.  Every wait of a thread block for its
 * neighbours is bounded (default 4 s): past the limit the block raises the
 * device error flag and returns, the other blocks see the flag and return
 * too, and the host reads BDECON_ERR_TIMEOUT at the next sync; the CUDA
 * context stays usable.  silent_block >= 0 makes that block of the sweep
 * kernel never publish its progress, so its neighbours' waits run out;
 * wait_ns sets the wait limit (1 ms .. 60 s).  silent_block = -1 restores
 * normal operation.                                                        */
bdecon_status bdecon_set_fault(bdecon_handle* h, int32_t silent_block, int64_t wait_ns);

/* Per-kernel timing: while enabled, CUDA events on the handle's stream
 * bracket every launch of the sweep kernel.  bdecon_sweep_kernel_time
 * synchronises, returns the summed device time (ms) and the number of
 * launches measured since the last call, and resets both.                  */
bdecon_status bdecon_set_timing(bdecon_handle* h, int32_t enable);
bdecon_status bdecon_sweep_kernel_time(bdecon_handle* h, double* ms, int64_t* launches);

/* ---------------------------------------------------------------- serving */

/* A serving loop with continuous batching: a library thread admits queued
 * jobs (one problem each) when a job slot is free and the job's device
 * workspace fits the memory budget, sweeps all running jobs together (per segment
 * of at most segment_sweeps sweeps, one cooperative launch per group of
 * jobs sharing PSF side, stride and update team, or one over every job), and between segments
 * retires finished jobs -- keeping their posterior mean for polling -- and
 * admits new ones.  Chain state stays resident on the device while a job
 * runs.  A job's chains use their own sweep counter, refresh schedule and
 * random stream, so each result is bit-identical to the same job run alone.
 * Errors of submit/poll/wait are reported through bdecon_last_error(NULL). */
typedef struct bdecon_server bdecon_server;

typedef struct {
    size_t mem_budget;         /* device bytes for the running jobs' workspaces     */
    int32_t max_jobs;          /* jobs running at once, >= 1                         */
    int32_t segment_sweeps;    /* sweeps per shared segment, 1..64                  */
    int32_t precision;         /* bdecon_precision of every job                      */
    int32_t device;            /* CUDA device ordinal                                */
    int32_t one_launch;        /* 1: one launch over every running job per segment   */
} bdecon_server_config;

typedef enum {
    BDECON_JOB_QUEUED = 0,
    BDECON_JOB_RUNNING = 1,
    BDECON_JOB_DONE = 2,
    BDECON_JOB_FAILED = 3
} bdecon_job_state;

/* Start the server thread on its own CUDA stream.                          */
bdecon_status bdecon_server_start(const bdecon_server_config* cfg, bdecon_server** out);

/* Queue a job of `sweeps` sweeps, more than its burn_in (inputs are copied;
 * max_sweeps and flags of the problem are replaced).  A job whose workspace exceeds the budget is
 * marked failed at once.                                                    */
bdecon_status bdecon_server_submit(bdecon_server* s, const bdecon_problem* job, int32_t sweeps,
                                   int64_t* job_id);

/* State of a job; times (optional, 3 doubles, seconds on the host's steady
 * clock) = submit, start, finish; when done and mean is non-NULL, the
 * posterior mean over all its chains, (H+2R)*(W+2R) doubles (cap = capacity
 * in doubles).  BDECON_ERR_STATE for a failed job.                          */
bdecon_status bdecon_server_poll(bdecon_server* s, int64_t job_id, int32_t* state, double* times,
                                 double* mean, size_t cap);

/* Block until the job is done or failed, or timeout_s elapses.             */
bdecon_status bdecon_server_wait(bdecon_server* s, int64_t job_id, double timeout_s, int32_t* state);

bdecon_status bdecon_server_stats(bdecon_server* s, int64_t* queued, int64_t* running, int64_t* done,
                                  size_t* mem_used, int64_t* segments);

/* Stop: queued jobs fail, the running segment completes, running jobs fail,
 * all device memory of the server and its jobs is freed.                    */
bdecon_status bdecon_server_stop(bdecon_server* s);

/* ----------------------------------------------------- allocation-free */

/* Log posterior of Eq. 9 (the same quantity as bdecon_log_posterior) for an
 * object held in device memory, without allocating any device memory.  The
 * paper has no counterpart to this entry point: it exists for callers that
 * must not call cudaMalloc or cudaFree once running -- for example an
 * acquisition loop that reserved all device memory for frame buffers up
 * front, or a host whose device allocator belongs to another framework and
 * forbids outside allocations and the device synchronisation they can
 * cause.  Creating a handle allocates, so such callers cannot use
 * bdecon_log_posterior.
 *
 * Arguments mirror bdecon_problem, but every array is a DEVICE pointer:
 * image, gain_map, offset_map, var_map (H*W float, maps may be NULL to use
 * the scalar), psf (L*L double, >= 0, sum > 0; normalised here), rho
 * ((H+2R)*(W+2R) double, > 0) and out (one double, written on the stream).
 * Input values are not checked on the host (that would need a copy);
 * invalid values give a non-finite result.  Work is queued on stream
 * (cudaStream_t or NULL); the call returns without waiting.
 *
 * Scratch comes from one fixed array of 2^19 = 524288 doubles (4 MiB) in
 * the library's device memory, held by every GPU that loads the library
 * until the process exits.  A problem needs L*L + 5*S*S + ceil(H*W/256) +
 * ceil((H+2R)/S)*ceil((W+2R)/S) doubles (S the stride, L when 0); one
 * needing more than 2^19 is refused with BDECON_ERR_INVALID and a message
 * from bdecon_last_error(NULL).  The limit therefore depends on the stride:
 * about 32 megapixels at S = L = 9, 70 at S = L = 17, 4.5 at S = L = 3 and
 * 0.5 at S = L = 1.  The first call on each device looks up the array's
 * device address (once per device, with that device current).  Under the
 * CUDA runtime's lazy module loading (the default) that first lookup may
 * also load the library's device code and, with it, place the 4 MiB array:
 * a one-time reservation made by the CUDA runtime, not by this call.  A
 * caller that cannot allow even that while running makes one call during
 * its set-up; that first call should also come before any stream capture.
 * Later calls allocate nothing.  All calls share the array and it keeps
 * the last call's contents (each call clears what it accumulates into):
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialised by the caller.                         */
bdecon_status bdecon_log_posterior_static(int32_t H, int32_t W, const float* image, int32_t L,
                                          const double* psf, const float* gain_map, double gain,
                                          const float* offset_map, double offset,
                                          const float* var_map, double read_var, int32_t stride,
                                          const double* rho, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BDECON_H */
