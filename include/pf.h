/*
 * pf.h -- C ABI of the GB300 particle-learning library (libpf.so).
 *
 * Implements one full particle-learning cycle of McAlinn & Nakatsuma,
 * "Parallel Resampling for Fully Parallelized Particle Filters"
 * (arXiv 1212.1639): predictive-likelihood weights, the resampling CDF,
 * parallel resampling against that CDF, and propagation of the state and its
 * conjugate sufficient statistics (paper Section 2, Algorithm "Particle
 * Learning"; Section 3, resampling; Section 4, the local-level model
 *   y_t = x_t + v_t, v_t ~ N(0, sigma^2);  x_t = x_{t-1} + w_t, w_t ~ N(0, tau^2)
 * with inverse-gamma priors on sigma^2 and tau^2).
 *
 * Every step runs on the GPU (sm_103a).  Host <-> device traffic is limited to
 * the observations going in and summaries coming out (paper Section 3.2,
 * closing paragraph: transfers only at the edges).
 *
 * Conventions
 *  - All functions return a pf_status; none throws or exits.  On failure
 *    pf_last_error() returns a thread-local message.
 *  - A filter handle owns all of its device memory.  A handle is not
 *    thread-safe; distinct handles are independent.
 *  - A CUDA error or a device error word (lookback timeout, non-finite
 *    weights, a gamma sampler that rejected 16 times) makes the handle
 *    sticky-failed: every later call except pf_destroy returns that status.
 *  - Calls are asynchronous on the handle's stream unless stated otherwise;
 *    device errors surface at the next synchronising call (pf_estimate,
 *    pf_sync, pf_get_*).
 *  - Pointers documented as "host or device" may be either (the copy uses
 *    unified addressing).
 *  - Random draws are addressed by (seed, filter_id, t, particle, purpose):
 *    counter-based Philox4x32-10, so results do not depend on launch shapes.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PF_OK = 0,
  PF_ERR_INVALID = 1,  /* bad argument (NULL, n out of range, bad enum, a0 < 1) */
  PF_ERR_OOM = 2,      /* device or pinned allocation failed */
  PF_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  PF_ERR_NUMERIC = 4,  /* non-finite or negative weights, all-zero CDF, gamma sampler failure */
  PF_ERR_TIMEOUT = 5,  /* a bounded device wait (scan lookback) gave up */
  PF_ERR_BUSY = 6      /* admission refused (memory budget) */
} pf_status;

/* Resampling scheme (paper Section 3.1).  All schemes draw ancestors from the
 * same exact integer CDF Q (Q_i = sum_{l<=i} W_l, T = Q_{n-1}); slot j's
 * ancestor is the first i with Q_i > position_j.
 *  MULTINOMIAL            positions = order statistics of n iid uniforms on
 *                         [0, T), generated in ascending order (exponential
 *                         spacings), matched to the CDF by a merge.
 *  SYSTEMATIC             positions = (j + u0) T / n, one uniform u0.
 *  MULTINOMIAL_CUTPOINT   same positions as MULTINOMIAL, searched with the
 *                         paper's parallelized cut-point search and cut-point
 *                         method (Section 3.2); identical output.
 *  SYSTEMATIC_CUTPOINT    same positions as SYSTEMATIC, cut-point search.
 *                         In the cut-point search thread i writes the whole
 *                         run of table entries that point at particle i, as
 *                         the paper's algorithm does; under degenerate
 *                         weights (one particle holding nearly all the mass,
 *                         the worst case Section 3.2 discusses) one thread
 *                         writes up to n entries serially, so both
 *                         *_CUTPOINT schemes take O(n) time there.  The
 *                         other schemes have no such case.
 *  STRATIFIED             positions = (j + u_j) T / n, one uniform u_j in
 *                         each stratum (Section 3.1, "Stratified
 *                         Resampling"): u_j from word pair 2 (j mod 2),
 *                         2 (j mod 2) + 1 of the draw (seed, filter, t,
 *                         floor(j/2), purpose 9).  Single filters and
 *                         pf_resample; the batched and served forms take
 *                         the first four schemes.
 * Ancestors come out in nondecreasing order (the sorted expansion of the
 * offspring counts). */
typedef enum {
  PF_MULTINOMIAL = 0,
  PF_SYSTEMATIC = 1,
  PF_MULTINOMIAL_CUTPOINT = 2,
  PF_SYSTEMATIC_CUTPOINT = 3,
  PF_STRATIFIED = 4
} pf_scheme;

/* State precision (the paper's GPU(sp) and GPU(dp) modes, Section 4).
 * FP32: x, sigma^2, tau^2 in binary32, sufficient statistics as exact 64-bit
 *       fixed point (2^-32 units), log marginal likelihood accumulated in
 *       binary64 from an exact 128-bit fixed-point particle sum.
 * FP64: everything in binary64. */
typedef enum { PF_FP32 = 0, PF_FP64 = 1 } pf_precision;

/* Optional device allocator (e.g. a caching allocator).  alloc returns NULL on
 * failure.  stream is the handle's cudaStream_t. */
typedef void* (*pf_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pf_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
  uint64_t n_particles;    /* 1 .. PF_MAX_PARTICLES */
  uint64_t seed;           /* Philox key */
  uint32_t filter_id;      /* third Philox counter word: independent streams per filter */
  int32_t scheme;          /* pf_scheme */
  int32_t precision;       /* pf_precision */
  int32_t known_variances; /* nonzero: sigma^2, tau^2 fixed (no learning; Kalman check) */
  double x0_mean, x0_var;  /* x_0 ~ N(x0_mean, x0_var) */
  double a_sigma, b_sigma; /* sigma^2 ~ IG(a_sigma, b_sigma), shape/scale, a_sigma >= 1 */
  double a_tau, b_tau;     /* tau^2 ~ IG(a_tau, b_tau), a_tau >= 1 */
  double sigma2, tau2;     /* used when known_variances != 0 */
  void* stream;            /* cudaStream_t; NULL = legacy default stream */
  pf_alloc_fn alloc;       /* NULL: cudaMallocAsync / cudaFreeAsync on stream */
  pf_free_fn free;
  void* alloc_ctx;
  int32_t algorithm;       /* pf_algorithm; 0 = particle learning */
  /* Adaptive resampling (particle learning, single filters; not in the
   * paper, which resamples every cycle).  0: resample every cycle.  In
   * (0, 1]: the filter carries log-weights lambda_i between cycles, combines
   * them with the predictive weights (L_i = lambda_i + log p(y | z_i)) and
   * resamples only when ESS = (sum W)^2 / sum W^2 of the quantised weights
   * is below ess_frac * n_particles (decided in binary64 from the exact
   * integer sums); otherwise every particle is its own ancestor and carries
   * lambda_i = L_i - max L.  The log marginal likelihood is normalised by
   * sum exp(lambda) and the summaries are weighted by exp(lambda). */
  double ess_frac;
} pf_config;

/* The cycle run by a single filter.
 *  PARTICLE_LEARNING  Algorithm "Particle Learning" (Section 2): resample
 *                     with p(y_{t+1} | z_t), propagate x conditional on
 *                     y_{t+1}, update the sufficient statistics, draw theta.
 *  BOOTSTRAP          Algorithm "Particle Filtering" (Section 2) with the
 *                     variances known (known_variances != 0 required):
 *                     propagate x_t ~ N(x~_{t-1}, tau^2) (Box-Muller's first
 *                     output of the draw (seed, filter, t, i, purpose 10)),
 *                     weight by p(y_t | x_t) = N(y_t; x_t, sigma^2),
 *                     resample.  Same CDF, resampling schemes, summaries and
 *                     log marginal likelihood estimate.  Single filters only. */
typedef enum { PF_PARTICLE_LEARNING = 0, PF_BOOTSTRAP = 1 } pf_algorithm;

#define PF_MAX_PARTICLES (1ull << 26)

/* Posterior summaries after t observations (paper Section 2, the paragraph
 * after Algorithm "Particle Learning": posterior statistics of theta from the
 * particles).  Means and population variances over the particles; the log
 * marginal likelihood log p(y_1..y_t) is the particle estimate
 * sum_s [ log (1/n) sum_i p(y_s | z_{s-1}^(i)) ]. */
typedef struct {
  uint64_t t;
  double x_mean, x_var;
  double sigma2_mean, sigma2_var;
  double tau2_mean, tau2_var;
  double log_marglik;
} pf_estimates;

typedef struct pf_filter pf_filter;

/* Create a filter and enqueue its initialisation (Algorithm "Particle
 * Learning", Step 0: x_0, sigma^2, tau^2 drawn from the priors).  *out
 * receives the handle.  Errors: PF_ERR_INVALID, PF_ERR_OOM, PF_ERR_CUDA. */
pf_status pf_create(const pf_config* cfg, pf_filter** out);

/* Enqueue one cycle for observation y = y_{t+1} (Steps 1-4): weights
 * w_i ~ p(y | z_t^(i)), the CDF, resampling, propagation of x, update of the
 * sufficient statistics, draw of sigma^2 and tau^2.  Asynchronous.
 * After pf_step_ahead(f, y', y_next), y must equal y_next bit for bit
 * (else PF_ERR_INVALID, nothing enqueued, the handle stays usable). */
pf_status pf_step(pf_filter* f, double y);

/* Enqueue one cycle for observation y, as pf_step, whose propagation (Steps
 * 2-4) also computes the next cycle's Step 1 weights w_j ~ p(y_next | z_{t+1}^(j))
 * and their maximum while each new particle is still in registers, so the next
 * cycle skips the weights kernel and its re-read of the state.  Results are
 * bit for bit those of pf_step(y) followed by pf_step(y_next).  The next
 * pf_step / pf_step_ahead / pf_step_profiled call on this handle must pass
 * y_next as its observation (bitwise; else PF_ERR_INVALID, nothing enqueued).
 * The first call on a handle captures the fused cycle forms as CUDA graphs on
 * the handle's stream (make it outside any stream capture).  Bootstrap filters
 * (PF_BOOTSTRAP) weigh after their own blind propagation: for them this is
 * pf_step(f, y).  Asynchronous. */
pf_status pf_step_ahead(pf_filter* f, double y, double y_next);

/* Enqueue n_steps cycles for the observations y[0..n_steps) (host or device
 * pointer, binary64): n_steps calls of pf_step.  Replays a CUDA graph of one
 * cycle; each launch carries its observation in the graph's weights-node
 * arguments: a host value by value, a device observation by address, read
 * when the cycle runs (so a device buffer must stay valid until the cycles
 * have run, in stream order).  With device-resident observations,
 * PF_ERR_INVALID if a pf_step_ahead announcement is pending (it cannot be
 * compared on the host). */
pf_status pf_run(pf_filter* f, const double* y, uint32_t n_steps);

/* Reduce the particles to posterior summaries (paper Section 2) and copy
 * them to *out (host).  Synchronises the handle's stream. */
pf_status pf_estimate(pf_filter* f, pf_estimates* out);

/* One cycle for observation y and its posterior summaries in *out (host):
 * pf_step(f, y) followed by pf_estimate(f, out) with the same results, as
 * one captured graph (the cycle, the summary reduction and a 104-byte copy
 * to pinned host memory) and one synchronisation.  For a caller that reads
 * the filter's result after every observation.  Synchronises. */
pf_status pf_step_estimate(pf_filter* f, double y, pf_estimates* out);

/* Wait for all enqueued work and check the device error word. */
pf_status pf_sync(pf_filter* f);

/* Measurement: run one cycle exactly as pf_step does, but with each kernel
 * launched on its own (no graph) and bracketed by CUDA events on the
 * handle's stream.  Writes up to max_kernels kernel durations in
 * milliseconds to kernel_ms (host), their static names to kernel_names (host,
 * may be NULL) and the count to *n_kernels.  Synchronises. */
pf_status pf_step_profiled(pf_filter* f, double y, float* kernel_ms, const char** kernel_names,
                           int max_kernels, int* n_kernels);

/* Measurement: pf_step_ahead(f, y, y_next) with each kernel launched on its
 * own between CUDA events, as pf_step_profiled.  Synchronises. */
pf_status pf_step_ahead_profiled(pf_filter* f, double y, double y_next, float* kernel_ms,
                                 const char** kernel_names, int max_kernels, int* n_kernels);

/* Copy the current particles out (paper Section 4, "Store": optional).
 * Buffers are host or device; NULL skips an array.  FP32 filters write
 * float x/sigma2/tau2 and uint64 fixed-point (2^-32) b_sigma/b_tau; FP64
 * filters write doubles.  Synchronises. */
pf_status pf_get_particles(pf_filter* f, void* x, void* sigma2, void* tau2, void* b_sigma,
                           void* b_tau);

/* Copy the last cycle's ancestor indices (n uint32, host or device) and,
 * if Q is not NULL, its CDF (n uint64).  With adaptive resampling, a cycle
 * that did not resample has the identity as its ancestors (its CDF is still
 * that of the combined weights).  Synchronises. */
pf_status pf_get_ancestors(pf_filter* f, uint32_t* anc, uint64_t* Q);

/* Free every device buffer of the handle (after the stream's pending work).
 * NULL-safe. */
pf_status pf_destroy(pf_filter* f);

/* Checkpoint and resume.  The paper runs each series in one go; a long-lived
 * filter (a service restarting, a job moving to another GPU) needs its state
 * saved and continued.  A checkpoint holds the filter's configuration (model,
 * priors, seed, filter id, scheme, precision, algorithm), the number of
 * cycles t, the accumulated log marginal likelihood and every particle's x,
 * sigma^2, tau^2, b_sigma, b_tau.  Resuming draws the same Philox counters
 * (seed, filter, t, particle, purpose), so the restored filter continues bit
 * for bit as the original would have.  The blob is self-describing (magic,
 * format version, sizes) and valid for this library version.
 *
 * pf_checkpoint_size: *bytes receives the blob size for this handle. */
pf_status pf_checkpoint_size(pf_filter* f, size_t* bytes);

/* Write the checkpoint to buf (host or device memory, at least
 * pf_checkpoint_size bytes; the caller owns it).  Synchronises the handle's
 * stream first.  PF_ERR_INVALID if bytes is too small or if a pf_step_ahead
 * announcement is pending (its precomputed weights are not saved: pass the
 * announced observation to pf_step first); sticky errors as usual. */
pf_status pf_checkpoint(pf_filter* f, void* buf, size_t bytes);

/* Create a filter from a checkpoint (host or device memory, `bytes` long).
 * The model, sizes, seed and scheme come from the checkpoint; cfg (may be
 * NULL) supplies only stream, alloc, free and alloc_ctx, with the meaning
 * they have in pf_create.  Synchronises the new handle's stream before
 * returning.  PF_ERR_INVALID for a blob that is truncated, of another format
 * version or not a checkpoint; PF_ERR_OOM / PF_ERR_CUDA as pf_create. */
pf_status pf_restore(const pf_config* cfg, const void* buf, size_t bytes, pf_filter** out);

/* Thread-local description of the last failure on this thread. */
const char* pf_last_error(void);

/* Resampling alone (paper Section 3): quantise the n binary32 weights
 * w_dev[0..n) (nonnegative, not all zero; need not be normalised) to the
 * exact CDF, W_i = floor(w_i 2^(k-e)) with k = 61 - ceil(log2 n) and
 * max_i w_i = f 2^e, f in [1/2, 1), and write n ancestor indices to anc_dev
 * (nondecreasing).  Draws use (seed, filter_id, t).  Device pointers on
 * `stream` (cudaStream_t, may be NULL); the call borrows them.  Scratch is
 * allocated on the stream from a stream-ordered memory pool that the library
 * owns (one per device, created on first use; it keeps up to 256 MiB of freed
 * scratch for later calls) and freed before the call returns.  Errors: PF_ERR_INVALID (NULL, n out of range, bad scheme);
 * PF_ERR_NUMERIC (a negative / non-finite weight or all zero), detected on
 * the device and reported after a stream synchronisation, which this call
 * performs. */
pf_status pf_resample(const float* w_dev, uint64_t n, uint64_t seed, uint32_t filter_id,
                      uint32_t t, int32_t scheme, uint32_t* anc_dev, void* stream);

/* The exact fixed-point resampling CDF of eq. (resample.cdf) for binary32
 * weights: Q_dev[i] = sum_{l<=i} W_l (uint64), W as in pf_resample.  Device
 * pointers; synchronises.  Errors as pf_resample. */
pf_status pf_cdf(const float* w_dev, uint64_t n, uint64_t* Q_dev, void* stream);

/* Algorithm "Parallelized Cut-Point Search" (paper Section 3.2) on a finished
 * CDF Q_dev[0..n) (nondecreasing, Q_{n-1} = T > 0, T <= 2^62): writes the
 * cut-points I_dev[k] = min{i : Q_i / T > k / n}, k = 0..n-1 (0-based), via
 * L_i = ceil(n Q_i / T).  Device pointers; synchronises. */
pf_status pf_cutpoint_search(const uint64_t* Q_dev, uint64_t n, uint32_t* I_dev, void* stream);

/* Algorithm "Parallelized Cut-Point Method" (paper Section 3.2) for explicit
 * integer positions U_dev[0..m) in [0, T): thread j starts at
 * I_{floor(n U_j / T)} and climbs while Q_k <= U_j; anc_dev[j] = k.
 * Device pointers; synchronises. */
pf_status pf_cutpoint_method(const uint64_t* Q_dev, uint64_t n, const uint32_t* I_dev,
                             const uint64_t* U_dev, uint64_t m, uint32_t* anc_dev,
                             void* stream);

/* Resampling without allocating: the same computation and result as
 * pf_resample, for callers that cannot allocate device memory at the point
 * where they resample: latency-critical loops that must not risk an
 * allocation's synchronisation, or processes whose device memory is reserved
 * up front and must not grow.  It avoids device allocation only: the call
 * still makes CUDA runtime calls (cudaGetDevice, cudaMemsetAsync, kernel
 * launches, a small cudaMemcpyAsync) and synchronises `stream` before it
 * returns, so it may not be called from a host function enqueued on a stream
 * (where CUDA API calls are forbidden).  The paper has no counterpart; this is
 * a deployment variant.
 *
 * Scratch lives in one fixed-size device array inside libpf.so, present on
 * every device that loads the library until the process exits (about 20 MiB),
 * and sized for n <= PF_NOALLOC_MAX_PARTICLES; larger n returns
 * PF_ERR_INVALID.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current.  The device used is
 * the calling thread's current device, which must be the one that holds
 * w_dev and anc_dev.  Every call on a device shares the one array, so calls
 * whose GPU work overlaps (other streams, other host threads) race and
 * corrupt each other: serialise them.  The call clears the parts of the
 * scratch that must start at zero, then synchronises `stream` to report
 * device-side errors as pf_resample does.  Arguments and errors as
 * pf_resample. */
#define PF_NOALLOC_MAX_PARTICLES (1ull << 20)
pf_status pf_resample_noalloc(const float* w_dev, uint64_t n, uint64_t seed, uint32_t filter_id,
                              uint32_t t, int32_t scheme, uint32_t* anc_dev, void* stream);

/* ---------------------------------------------------------------------------
 * Batched filters: many independent particle-learning filters of uneven size
 * advanced together, one persistent kernel launch per cycle (replayed from a
 * CUDA graph).  Each CTA of the launch takes whole filters from a work list
 * ordered by size, largest first, and runs the full cycle of the paper's
 * Algorithm "Particle Learning" (Steps 1-4) for each with block barriers
 * only.  The paper runs one filter at a time; batching is a deployment
 * variant of the same cycle.
 *
 * Every filter of a batch gives bit for bit the results of a standalone
 * pf_create filter with the same pf_config: the same ancestors, particles,
 * summaries and log marginal likelihood.
 *
 * Particles of all filters live in one device pool sized at creation (the
 * HBM budget); filters are admitted into slots while the pool and the slots
 * have room (first fit, 32-particle granules) and leave with
 * pf_batch_remove.  Scheme and precision are shared by the whole batch.
 * --------------------------------------------------------------------------- */
typedef struct pf_batch pf_batch;

typedef struct {
  uint32_t max_filters;      /* slots; 0 = the number of initial filters */
  uint64_t hbm_budget_bytes; /* device bytes for the particle pool; 0 = exactly
                                what the initial filters need */
  int32_t scheme;            /* pf_scheme of every filter (the cut-point variants
                                give the same ancestors as their base schemes) */
  int32_t precision;         /* pf_precision of every filter */
  int32_t autotune;          /* nonzero: the first pf_batch_step runs pf_batch_tune */
  void* stream;              /* cudaStream_t; NULL = a stream the batch creates */
  pf_alloc_fn alloc;         /* NULL: cudaMallocAsync / cudaFreeAsync */
  pf_free_fn free;
  void* alloc_ctx;
  int32_t adaptive;          /* nonzero: the pool also holds each particle's carried
                                log-weight (one more value per particle), so that
                                filters may set ess_frac > 0 (adaptive resampling) */
} pf_batch_opts;

typedef struct {
  uint32_t max_filters, resident;       /* slots, slots in use */
  uint64_t pool_particles;              /* pool capacity */
  uint64_t used_particles;              /* taken by resident filters (rounded to granules) */
  uint64_t bytes_per_particle;          /* device bytes per pool particle */
  uint64_t pool_bytes;
  uint32_t grid, block;                 /* persistent launch shape of the cycle kernel */
  uint32_t cluster;                     /* CTAs per cluster (1: no clusters) */
  uint32_t big_min;                     /* clusters take filters of at least this many particles */
  uint32_t tuned;                       /* nonzero once pf_batch_tune or pf_batch_set_shape chose it */
  uint64_t cycles;                      /* pf_batch_step calls that launched work */
} pf_batch_info;

/* Launch shapes timed by pf_batch_tune. */
#define PF_BATCH_MAX_SHAPES 16
typedef struct {
  uint32_t n_shapes;
  uint32_t block[PF_BATCH_MAX_SHAPES];  /* threads per CTA */
  uint32_t grid[PF_BATCH_MAX_SHAPES];   /* CTAs of the persistent launch */
  uint32_t cluster[PF_BATCH_MAX_SHAPES];  /* CTAs per cluster */
  uint32_t big_min[PF_BATCH_MAX_SHAPES];  /* filter size from which a whole cluster takes it */
  float ms[PF_BATCH_MAX_SHAPES];        /* mean trial cycle time */
  uint32_t chosen;                      /* index of the shape kept */
} pf_batch_tuning;

/* Create a batch with n initial filters cfgs[0..n) (host array, may be NULL
 * when n = 0) in slots 0..n-1, and enqueue their initialisation (Step 0).
 * Per filter, cfgs[i] supplies n_particles, seed, filter_id, the priors,
 * known-variance settings and ess_frac (> 0 only in a batch created with
 * adaptive != 0); its scheme and precision must equal opts'; its algorithm
 * must be particle learning; its stream and allocator fields are ignored.  Errors: PF_ERR_INVALID,
 * PF_ERR_OOM, PF_ERR_CUDA, PF_ERR_BUSY (the budget cannot hold the initial
 * filters).  The initialisation runs asynchronously on the batch's stream. */
pf_status pf_batch_create(const pf_config* cfgs, uint32_t n, const pf_batch_opts* opts,
                          pf_batch** out);

/* Admit one more filter: the lowest free slot goes to *slot and its
 * initialisation is enqueued (asynchronous; it does not wait for cycles in
 * flight).  PF_ERR_BUSY when no slot is free or no free pool range holds
 * cfg->n_particles (nothing changes then). */
pf_status pf_batch_add(pf_batch* b, const pf_config* cfg, uint32_t* slot);

/* Release a slot and its pool range (reused only by work enqueued later on
 * the batch's stream).  PF_ERR_INVALID for a slot not in use. */
pf_status pf_batch_remove(pf_batch* b, uint32_t slot);

/* Enqueue one cycle for the resident filters s with mask[s] != 0 (mask NULL:
 * every resident filter), filter s consuming observation y[s].  y and mask
 * are host arrays indexed by slot (max_filters entries).  Asynchronous: one
 * host-to-device copy of the work list (16 bytes per stepped filter) and one
 * graph launch. */
pf_status pf_batch_step(pf_batch* b, const double* y, const uint8_t* mask);

/* Autotuner: time the cycle of the selected filters (y, mask as in
 * pf_batch_step) under every candidate launch shape and keep the fastest for
 * later cycles.  Candidates: one CTA per filter with 256 or 512 threads and 1
 * up to the resident maximum of CTAs per SM; and thread-block clusters of 2,
 * 4 or 8 CTAs of 256 threads, where filters of at least 1 or 4 scan tiles
 * (4096 particles) per CTA of the cluster are processed by a whole cluster
 * together (exchanging their scan totals through distributed shared memory)
 * and smaller ones by single CTAs.  The trial cycles commit nothing (t, the log marginal
 * likelihood and the error words are unchanged; the next pf_batch_step
 * overwrites every buffer they wrote), and the launch shape never changes a
 * result.  *out (may be NULL) receives the timings.  Synchronises. */
pf_status pf_batch_tune(pf_batch* b, const double* y, const uint8_t* mask, pf_batch_tuning* out);

/* Fix the launch shape instead of tuning: block 256 or 512 threads per CTA
 * without clusters (cluster 0 or 1), or 256 threads in clusters of 2, 4 or 8
 * CTAs, which take the filters of at least big_min particles together; grid
 * a multiple of the cluster size up to the resident maximum for the shape
 * (any count works: CTAs and clusters take filters from the work list until
 * it is empty).  Counts as tuned.  Synchronises.  PF_ERR_INVALID for an
 * unsupported shape. */
pf_status pf_batch_set_shape(pf_batch* b, uint32_t block, uint32_t grid, uint32_t cluster,
                             uint32_t big_min);

/* Posterior summaries of the resident filters selected by mask (NULL: all),
 * written to out[slot] (host array of max_filters entries; other entries are
 * left alone).  Synchronises.  Returns the error of the first selected filter
 * whose device error word is set (PF_ERR_NUMERIC); its summaries are still
 * written. */
pf_status pf_batch_estimate(pf_batch* b, const uint8_t* mask, pf_estimates* out);

/* Wait for the batch's enqueued work. */
pf_status pf_batch_sync(pf_batch* b);

/* Copy one filter's particles (as pf_get_particles) or its last cycle's
 * ancestors and CDF (as pf_get_ancestors).  Buffers host or device; NULL
 * skips an array.  Synchronise. */
pf_status pf_batch_get_particles(pf_batch* b, uint32_t slot, void* x, void* sigma2, void* tau2,
                                 void* b_sigma, void* b_tau);
pf_status pf_batch_get_ancestors(pf_batch* b, uint32_t slot, uint32_t* anc, uint64_t* Q);

/* Occupancy of the pool and slots, and the launch shape.  Host only. */
pf_status pf_batch_get_info(pf_batch* b, pf_batch_info* out);

/* Free the batch after its stream's pending work.  NULL-safe. */
pf_status pf_batch_destroy(pf_batch* b);

/* ---------------------------------------------------------------------------
 * Serving: streams of observations that arrive at any time, each stream a
 * particle-learning filter whose state stays on the device.  A worker thread
 * inside the library does continuous batching: every cycle it takes the
 * oldest pending observation of every resident stream that has one, runs
 * them as one batched cycle (the pf_batch kernel) followed by the summaries
 * of the stepped streams, and keeps up to max_inflight cycles on the device
 * while it forms the next cycle from what has arrived meanwhile.  Streams are
 * admitted in FIFO order while the pool (sized by the HBM budget) and the
 * slots have room; a stream that does not fit waits (its observations queue)
 * until others close.
 *
 * Each observation yields one result: the stream's posterior summaries after
 * that observation, bit for bit what a standalone filter with the stream's
 * configuration gives after the same observations, however the streams were
 * interleaved.  Latency is measured from the submit call to the moment the
 * worker sees the summaries on the host.
 *
 * Thread safety: open / submit / close / poll / stats may be called from any
 * threads; the handle serialises them.
 * --------------------------------------------------------------------------- */
typedef struct pf_server pf_server;

typedef struct {
  uint32_t max_streams;       /* slots (resident streams at most) */
  uint64_t hbm_budget_bytes;  /* device bytes of the particle pool (> 0) */
  int32_t scheme;             /* pf_scheme of every stream */
  int32_t precision;          /* pf_precision of every stream */
  uint32_t max_inflight;      /* cycles on the device at once, 1..4 (0 = 2) */
  int32_t keep_results;       /* nonzero: keep per-observation results for pf_server_poll */
  uint32_t block, grid;       /* launch shape (0 = the batch default) */
  uint32_t cluster, big_min;  /* clusters of CTAs for large streams (0 = none) */
  double warmup_s;            /* steady-state latency counts observations submitted this
                                 long after the first one */
  void* stream;               /* cudaStream_t; NULL = one the server creates */
  pf_alloc_fn alloc;          /* NULL: cudaMallocAsync / cudaFreeAsync */
  pf_free_fn free;
  void* alloc_ctx;
  int32_t adaptive;           /* as pf_batch_opts.adaptive: streams may set ess_frac > 0 */
} pf_server_opts;

typedef struct {
  uint64_t stream_id;
  uint64_t seq;              /* observation index within the stream, from 0 */
  pf_estimates est;          /* summaries after this observation */
  float latency_us;          /* submit -> summaries on the host */
  int32_t status;            /* PF_OK, or PF_ERR_NUMERIC if the filter's error word is set */
} pf_server_result;

typedef struct {
  uint64_t submitted, completed;        /* observations */
  uint64_t cycles, particle_steps;      /* batched cycles; sum of n over completed observations */
  uint64_t streams_opened, streams_closed, admitted, admitted_after_wait;
  uint32_t waiting, resident;           /* streams now waiting for admission / resident */
  uint64_t pool_particles, used_particles;
  double mean_cycle_streams;            /* streams per cycle */
  uint32_t max_cycle_streams;
  double mean_admission_wait_us, replay_max_lag_us;
  double wall_s;                        /* first submit -> last result */
  double particle_steps_per_s, obs_per_s;
  double mean_us, p50_us, p90_us, p99_us, max_us;  /* observation latency */
  uint64_t steady_count;                            /* observations after the warm-up window */
  double steady_p50_us, steady_p90_us, steady_p99_us;
  uint32_t grid, block, cluster;
} pf_server_stats;

/* Replay event kinds (pf_server_replay). */
#define PF_EVENT_OBS 0
#define PF_EVENT_CLOSE 1
#define PF_EVENT_OPEN 2

/* Create a server and start its worker thread.  Errors: PF_ERR_INVALID,
 * PF_ERR_OOM, PF_ERR_CUDA. */
pf_status pf_server_create(const pf_server_opts* opts, pf_server** out);

/* Open stream `id` (any caller-chosen unique value) with configuration cfg
 * (as for pf_batch_add: scheme and precision must be the server's).  The
 * stream enters the admission queue; it is initialised once admitted.
 * PF_ERR_BUSY if it can never fit the pool. */
pf_status pf_server_open(pf_server* s, uint64_t id, const pf_config* cfg);

/* Queue observation y for stream id (time-stamped now). */
pf_status pf_server_submit(pf_server* s, uint64_t id, double y);

/* Close stream id once its queued observations are done; its slot and pool
 * range then go to waiting streams. */
pf_status pf_server_close(pf_server* s, uint64_t id);

/* Load generator: a library thread replays count events at times t_s[i]
 * (seconds from this call, nondecreasing): kind[i] PF_EVENT_OBS submits y[i]
 * to stream ids[i], PF_EVENT_CLOSE closes it, PF_EVENT_OPEN opens it with
 * cfgs[ids[i]] (cfgs has n_cfgs entries).  The arrays are copied; the call
 * returns at once.  PF_ERR_BUSY while another replay runs. */
pf_status pf_server_replay(pf_server* s, uint64_t count, const double* t_s, const uint8_t* kind,
                           const uint64_t* ids, const double* y, const pf_config* cfgs,
                           uint64_t n_cfgs);

/* Wait (up to timeout_s) until the replay has finished and every submitted
 * observation has its result.  PF_ERR_TIMEOUT otherwise. */
pf_status pf_server_drain(pf_server* s, double timeout_s);

/* Move up to max finished results (in completion order) to out; *n gets the
 * count.  Results are kept only with opts.keep_results. */
pf_status pf_server_poll(pf_server* s, pf_server_result* out, uint32_t max, uint32_t* n);

/* Counters, throughput and latency percentiles so far. */
pf_status pf_server_get_stats(pf_server* s, pf_server_stats* out);

/* Stop the worker after the cycles in flight, free everything.  Observations
 * still queued are dropped.  NULL-safe. */
pf_status pf_server_destroy(pf_server* s);

#ifdef __cplusplus
}
#endif

#endif /* PF_H */
