/*
 * libhawkes: spatiotemporal Hawkes log-likelihood, gradient and cut-posterior
 * location resample on one NVIDIA GB300 (sm_103a).
 *
 * Model (Sec. 2.1, eqs. 2-4 of "Scaling Hawkes processes to one million
 * COVID-19 cases"), for events (t_i, x_i, y_i) sorted by time:
 *   lambda_i = max( sum_{j: t_j != t_i} mu phi2(r_ij; tau_x) phi1(t_i - t_j; tau_t)
 *                 + sum_{j: t_j < t_i} theta omega e^{-omega (t_i - t_j)} phi2(r_ij; h s_j),
 *                   1e-40 )
 *   Lambda_i = mu [Phi((t_N - t_i)/tau_t) - Phi(-t_i/tau_t)] + theta [1 - e^{-omega (t_N - t_i)}]
 *   ell      = sum_i ( log lambda_i - Lambda_i )
 * phi2 is the 2-D spherical Gaussian density, phi1 the 1-D Gaussian density,
 * Phi the standard normal CDF, t_N the largest event time and s_j the fixed
 * bandwidth scale of the source event's county (eq. 3; s_j = 1 gives eq. 2).
 * The 1e-40 floor is the clip of Sec. 2.3.1; a clipped row contributes
 * log(1e-40) and nothing to the gradient.  The gradient is the exact
 * derivative of ell with respect to (mu, tau_x, tau_t, theta, omega, h).
 *
 * Conventions
 *  - Every call returns a status (HAWKES_OK = 0 or a negative error code);
 *    no C++ exception crosses this interface.
 *  - The caller owns every pointer it passes.  Host arrays are copied before
 *    the call returns.  Device pointers (the *_async calls) must stay valid
 *    until the work queued on the context's stream has finished, and must be
 *    8-byte aligned (they point at doubles); a misaligned one is rejected
 *    with HAWKES_ERR_ARG before any work is queued.
 *  - Each call that does work opens an NVTX range named after the call, so
 *    Nsight timelines show the library's calls (no cost without a tool).
 *  - Units are the caller's (the test workloads use km and days); times must
 *    be > 0 and non-decreasing, every value finite.
 *  - A device-side failure (a bounded wait that gave up, a non-finite result)
 *    is latched in the context and returned by the next synchronous call.
 *  - One context is used by one host thread at a time.
 */
#ifndef HAWKES_H
#define HAWKES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hawkes_ctx hawkes_ctx;

/* Model parameters.  tau_x, tau_t, omega, h > 0; mu, theta >= 0. */
typedef struct {
    double mu;     /* background weight (mu_0) */
    double tau_x;  /* background spatial lengthscale */
    double tau_t;  /* background temporal lengthscale */
    double theta;  /* self-excitation weight (xi_0) */
    double omega;  /* excitation decay rate (1 / sigma_t) */
    double h;      /* excitation spatial bandwidth multiplier (sigma_x) */
} hawkes_params;

enum {
    HAWKES_OK = 0,
    HAWKES_ERR_ARG = -1,        /* bad argument: null pointer, size, range, value */
    HAWKES_ERR_UNSORTED = -2,   /* times not non-decreasing, or not > 0 */
    HAWKES_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    HAWKES_ERR_NONFINITE = -4,  /* a result was NaN or infinite */
    HAWKES_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up */
    HAWKES_ERR_OOM = -6,        /* device allocation failed */
    HAWKES_ERR_STATE = -7,      /* call out of order (e.g. no events set) */
    HAWKES_ERR_TOO_LARGE = -8,  /* size above the fixed limit of hawkes_loglik_grad_noalloc */
    HAWKES_ERR_IO = -9,         /* a file could not be written (autotuner cache) */
    HAWKES_ERR_BOUNDS = -10     /* HAWKES_DEBUG build: a device-side index check failed */
};

/* Flags for the log-likelihood calls. */
enum {
    /*
     * Pair terms in FP32 (SFU exp2), per-row and global sums in FP64.  FP32
     * flushes every term below 2^-126 to zero.  Two FP64 fix-ups keep the
     * result that of the exact sum: rows whose FP32 rate is within 10^9 n of
     * that floor are recomputed in FP64 (so a flushed term cannot move a row
     * across the 1e-40 clip), and a bound on what the flushed terms can move
     * each output is kept per row; where an output's summed bound exceeds
     * 1e-8 of its magnitude, the rows whose bound exceeds 1e-8 of that
     * magnitude divided by the row count are recomputed in FP64 (at normal
     * bandwidths none is; with bandwidths so small that every excitation
     * term underflows, most are).
     */
    HAWKES_F32 = 0,
    HAWKES_F64 = 1,      /* every pair term in FP64 (slow on GB300: reference path) */
    HAWKES_MODEL2 = 0,   /* source bandwidth h * s_j from the county scale (eq. 3) */
    HAWKES_MODEL1 = 2,   /* s_j = 1 for every event (eq. 2) */
    /*
     * FP32 path only: skip tiles of the pair sweep whose every term is
     * exactly 0 in FP32 (flushed to zero): pairs farther apart in time than
     * sqrt(128) tau_t sqrt(2 / log2 e) contribute no background, and sources
     * earlier by more than (128 + max_j(-2 log2 s_j)) / (omega log2 e)
     * contribute no excitation.  The result is the same as without the flag
     * (the skipped terms are exact zeros); only the work shrinks.
     */
    HAWKES_SKIP_UNDERFLOW = 4,
    /*
     * The background exactly as eq. 2 prints it: a time-only Gaussian with a
     * constant spatial density, mu phi1(t_i - t_j; tau_t) / A, where the
     * kernel listing of App. A writes 1/A as tau_x^-2, so tau_x^2 plays the
     * role of the domain area A.  Lambda_i is unchanged (the spatial factor
     * has unit mass over the domain), d ell / d tau_x reduces to the -2/tau_x
     * factor of the constant, and mu and tau_x enter only as mu / tau_x^2.
     * Without this flag the background is the space-time Gaussian
     * mu phi2(r; tau_x) phi1(dt; tau_t).  Combines with every other flag.
     */
    HAWKES_BG_TIME = 8,
    /*
     * FP32 path, whole sum only (no row window), space-time background:
     * evaluate only the pairs that can be nonzero in FP32.  Events are
     * ordered by location (a Morton curve) inside time windows cut between
     * distinct times (hawkes_set_spatial_window); tiles of 256 events in that
     * order whose every background and excitation term is provably an exact
     * FP32 zero against a tile of rows (by bounding boxes of the current
     * locations and time ranges, with 2 units of margin on each base-2
     * exponent) are skipped.  The rest is evaluated pair by pair with exact
     * tie and causality indicators, so the result is the full sum up to
     * FP32 summation order.  The first call after hawkes_set_events builds
     * the order on the host (synchronous: make it outside stream capture).
     * Not for batches, HAWKES_F64, HAWKES_BG_TIME or row windows
     * (HAWKES_ERR_ARG).
     */
    HAWKES_SKIP_SPATIAL = 16,
    /*
     * Evaluate the log-likelihood only (the paper's own computation, Sec.
     * 2.3 and App. A; the univariate Metropolis-Hastings sampler of Sec. 2.2
     * needs no gradient).  The FP32 sweep then forms two moment sums per row
     * instead of six.  The six gradient outputs are NaN.  Combines with every
     * other flag; with HAWKES_F64 or HAWKES_BG_TIME the full kernels run and
     * only the gradient is dropped.
     */
    HAWKES_LOGLIK_ONLY = 32
};

/* Human-readable name of a status code (static storage). */
const char* hawkes_strerror(int status);

/*
 * Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * on that device on which all work is queued, or NULL for a stream the
 * context creates and owns.  *out is set to NULL on failure.
 */
int hawkes_create(hawkes_ctx** out, int device, void* cuda_stream);

/* Free the context and its device memory (waits for queued work).  NULL is a no-op. */
void hawkes_destroy(hawkes_ctx* ctx);

/*
 * Load n events (n >= 1), replacing any previous set.
 *   t[n]             event times, > 0, non-decreasing (HAWKES_ERR_UNSORTED otherwise)
 *   x[n], y[n]       event locations, or both NULL (all zero until the first
 *                    hawkes_resample_locations)
 *   county[n]        county of each event, 0 <= county < n_counties
 *   county_scale[n_counties]  s_c > 0, the source bandwidth scale of eq. 3
 * Ties in t are allowed: tied events exchange neither background nor
 * excitation terms (indicators t_j != t_i and t_j < t_i of eqs. 2-3).
 */
int hawkes_set_events(hawkes_ctx* ctx, int64_t n, const double* t, const double* x,
                      const double* y, const int32_t* county, int32_t n_counties,
                      const double* county_scale);

/*
 * County polygons for the location resample, as triangles (a fan of each
 * convex polygon or any other partition).
 *   tri_county[n_tri]  county of each triangle, non-decreasing; every county
 *                      of hawkes_set_events needs triangles of positive total area
 *   tri_xy[6 n_tri]    vertices ax, ay, bx, by, cx, cy of each triangle (finite)
 * A county id out of range or out of order, a non-finite vertex, or a county
 * without positive area returns HAWKES_ERR_ARG and leaves no counties set.
 */
int hawkes_set_counties(hawkes_ctx* ctx, int32_t n_tri, const int32_t* tri_county,
                        const double* tri_xy);

/*
 * Cut-posterior step of Sec. 2.2: draw every event location uniformly in its
 * county, replacing the current locations.  Event i uses the Philox4x64-10
 * block with counter (i, iteration, 0, 0) and key (seed, stream): word 0
 * picks the county's triangle with probability proportional to area, words
 * 1-2 place a uniform point in it (square-root barycentric map).  The draw
 * is a pure function of (seed, stream, iteration, i, county) and is
 * bit-identical to the documented FP64 formula.  Queued on the context
 * stream; returns without waiting.
 */
int hawkes_resample_locations(hawkes_ctx* ctx, uint64_t seed, uint64_t stream,
                              uint64_t iteration);

/* Copy the current event locations to host arrays x[n], y[n] (synchronous). */
int hawkes_get_locations(hawkes_ctx* ctx, double* x, double* y);

/*
 * Log-likelihood and gradient over the rows [row_begin, row_end) (the row
 * window of Sec. 2.3.2's multi-GPU split: summing the windows of a partition
 * of [0, n) gives the whole; every window uses all n events as sources and
 * the global t_N).  Pass row_begin = 0, row_end = n for the whole sum.
 *   params     host pointer
 *   flags      HAWKES_F32 or HAWKES_F64, | HAWKES_MODEL1 for s_j = 1,
 *              | HAWKES_SKIP_UNDERFLOW, | HAWKES_BG_TIME, | HAWKES_SKIP_SPATIAL,
 *              | HAWKES_LOGLIK_ONLY (grad then receives NaN)
 *   loglik     host pointer to one double (ell)
 *   grad       host pointer to six doubles, d ell / d (mu, tau_x, tau_t, theta, omega, h)
 * Synchronous: returns after the result is on the host.
 */
int hawkes_loglik_grad(hawkes_ctx* ctx, const hawkes_params* params, uint32_t flags,
                       int64_t row_begin, int64_t row_end, double* loglik, double* grad);

/*
 * As hawkes_loglik_grad over all rows, but queued on the context stream
 * without host synchronisation, so it can be captured in a CUDA graph.
 *   d_params  device pointer to one hawkes_params (read when the work runs)
 *   d_out     device pointer to 7 doubles: ell, then the six partials
 * Errors detected on the device are latched in the context.
 */
int hawkes_loglik_grad_async(hawkes_ctx* ctx, const hawkes_params* d_params, uint32_t flags,
                             double* d_out);

/*
 * Per-row values for testing at full size: as hawkes_loglik_grad over all
 * rows, and also writes rows[9 n] (host) = for each row i: ell_i, the six
 * partials of ell_i, log lambda_i, Lambda_i.
 */
int hawkes_loglik_rows(hawkes_ctx* ctx, const hawkes_params* params, uint32_t flags,
                       double* out7, double* rows);

/*
 * Symmetric row-tile shards of one evaluation, for a split across GPUs (Sec.
 * 2.3.2 splits the rows of one log-likelihood over GPUs and gathers the
 * per-row results; this split keeps the sweep's symmetric shortcut, in which
 * each unordered pair's background term is formed once and added to both of
 * its rows).  Shard g of G sweeps the symmetric work list's row tiles
 * [bounds[g], bounds[g+1]) (hawkes_shard_bounds with the context's
 * hawkes_shard_tile_rows), which hold about 1/G of the pairs each.  A row's
 * six moment sums then collect terms from every shard that holds a later row,
 * so the ranks add their moment vectors (one all-reduce of 6 n doubles) and
 * each finalises from the sum.
 *
 * hawkes_shard_bounds (host only; no device is touched): row boundaries
 *   bounds[nshards + 1], bounds[0] = 0, bounds[nshards] = n, non-decreasing,
 *   each inner one a multiple of tile_rows, chosen so that the shards' pair
 *   counts (pairs (i, j < i) of their rows) are as equal as whole tiles allow.
 *   Shards may be empty when nshards exceeds the tile count.
 * hawkes_shard_tile_rows: rows per row tile of the context's sweep variant
 *   (HAWKES_ERR_ARG for a NULL context).
 * hawkes_shard_moments: queue shard `shard` of `nshards` and write its moment
 *   sums to d_moments[6 n] (device, caller-owned; six consecutive vectors of
 *   n doubles: SB, SBr, SBt, SE, SEt, SEq of every row, unnormalised, natural
 *   units; rows outside the shard hold the column part it adds to them).
 *   Flags as for hawkes_loglik_grad_async, FP32 path only (HAWKES_F64 and
 *   HAWKES_SKIP_SPATIAL give HAWKES_ERR_ARG).  The first call for a new
 *   (shard, nshards, sweep variant) builds that shard's work list
 *   (synchronous: make it outside stream capture); later calls only queue.
 * hawkes_finalize_moments: from d_moments[6 n] summed over all shards (device,
 *   read when the work runs), queue the per-row finalisation and the global
 *   reduction of the whole sum, and write ell and the six partials to d_out[7]
 *   (device).  Same flags and parameters as the shards'.  Errors detected on
 *   the device are latched in the context.
 */
int hawkes_shard_bounds(int64_t n, int64_t tile_rows, int nshards, int64_t* bounds);
int64_t hawkes_shard_tile_rows(const hawkes_ctx* ctx);
int hawkes_shard_moments(hawkes_ctx* ctx, const hawkes_params* d_params, uint32_t flags,
                         int shard, int nshards, double* d_moments);
int hawkes_finalize_moments(hawkes_ctx* ctx, const hawkes_params* d_params, uint32_t flags,
                            const double* d_moments, double* d_out);

/* Timing of the context's kernels, accumulated while profiling is on. */
typedef struct {
    int64_t launches[8];   /* per kernel class (HAWKES_K_*) */
    double ms[8];          /* summed CUDA-event time of those launches */
} hawkes_profile;

enum {
    HAWKES_K_PREP = 0,     /* per-call FP32 staging of the event table */
    HAWKES_K_SWEEP = 1,    /* FP32 pair sweep */
    HAWKES_K_ROWS64 = 2,   /* FP64 pair rows */
    HAWKES_K_FINAL = 3,    /* per-row finalisation + block reduction */
    HAWKES_K_REDUCE = 4,   /* global reduction */
    HAWKES_K_RESAMPLE = 5, /* location resample */
    HAWKES_K_OTHER = 6     /* set-up kernels */
};

/*
 * Turn per-kernel CUDA-event timing on (1) or off (0); turning it on clears
 * the counters.  While on, every launch is bracketed by events on the
 * context stream (a small overhead); not for use under graph capture.
 */
int hawkes_profile_enable(hawkes_ctx* ctx, int on);

/* Wait for queued work and read the counters. */
int hawkes_profile_read(hawkes_ctx* ctx, hawkes_profile* out);

/*
 * Kernel variants of the FP32 pair sweep (rows per thread, resident CTAs per
 * SM).  All give the same result up to FP32 summation order; they differ in
 * speed by problem size.  hawkes_sweep_variants() is their number;
 * hawkes_set_sweep_variant selects one (synchronous; rebuilds the work list).
 */
int hawkes_sweep_variants(void);
int hawkes_set_sweep_variant(hawkes_ctx* ctx, int variant);
int hawkes_get_sweep_variant(const hawkes_ctx* ctx);

/*
 * Autotune the sweep on the current events: run every variant `reps` times
 * (after one warm-up) at `params` (host pointer; flags as for
 * hawkes_loglik_grad, FP32 path), time the sweep kernel with CUDA events,
 * keep the fastest.  *chosen receives its index; ms (optional, length
 * hawkes_sweep_variants()) the mean sweep time of each variant.
 */
int hawkes_tune(hawkes_ctx* ctx, const hawkes_params* params, uint32_t flags, int reps,
                int* chosen, double* ms);

/*
 * Autotuner cache.  A JSON file maps a configuration key to the tuned
 * choice, so that a process on a device and problem shape tuned before skips
 * the search.  The library writes the file as one JSON object with one entry
 * per line:
 *   {
 *   "<key>": {"variant": 0, "chunk": 16, "order": 0, "ms": 365.359, "nvariants": 5},
 *   ...
 *   }
 * The tuners below build the key as
 *   "<device name>|sm_<major><minor>|single|n<=2^<e>|flags=<flags>"
 *   "<device name>|sm_<major><minor>|batch|P=<P>|pairs<=2^<e>|flags=<flags>"
 * where 2^e is the smallest power of two >= n (single problem) or >= the
 * batch's total number of unordered pairs.  Entries written by a build with a
 * different number of sweep variants ("nvariants") are ignored, and lines
 * that do not parse are skipped, so a stale or damaged file only causes cache
 * misses.  Writes go to "<path>.tmp" and are renamed over the file.
 *
 * hawkes_tune_cached: look the context's key up in cache_path; on a hit,
 * select the cached variant (*from_cache = 1); on a miss, run hawkes_tune
 * (arguments as there) and store the result (*from_cache = 0).  *chosen
 * receives the variant.  Returns HAWKES_ERR_IO if the result was chosen but
 * could not be stored.
 */
int hawkes_tune_cached(hawkes_ctx* ctx, const hawkes_params* params, uint32_t flags, int reps,
                       const char* cache_path, int* chosen, int* from_cache);

/*
 * Host-only access to a cache file (no device is touched).
 *   hawkes_tune_cache_get: 1 if `key` has a valid entry (outputs, each
 *     optional, receive it), 0 if the file or the key is missing,
 *     HAWKES_ERR_ARG for a NULL path or a key containing '"', '\' or a
 *     control character.
 *   hawkes_tune_cache_put: insert or replace `key`; HAWKES_ERR_ARG for a bad
 *     key, a variant outside [0, hawkes_sweep_variants()), a negative chunk
 *     or order, or a negative or NaN time; HAWKES_ERR_IO if the file cannot
 *     be written.
 */
int hawkes_tune_cache_get(const char* cache_path, const char* key, int* variant, int* chunk,
                          int* order, double* ms);
int hawkes_tune_cache_put(const char* cache_path, const char* key, int variant, int chunk,
                          int order, double ms);

/*
 * Batched evaluation (many problems in one persistent launch).
 *
 * A batch groups P >= 1 contexts on one device, each with its own events
 * (MCMC chains with their own locations and parameters, or regional subsets
 * of uneven size).  One run resamples every problem's locations (if keys were
 * given), stages them, sweeps the pairs of ALL problems in a single
 * persistent kernel launch that takes work items (problem, row tile, column
 * chunk) from one queue, longest first, and reduces each problem to its own 7
 * outputs.  The paper ran its 30 chains as separate jobs (Sec. 3.2).
 *
 *   problems[P]        contexts with events set (and counties, if seeds are
 *                      given); each may appear once; the batch keeps pointers
 *                      to them, so destroy the batch before any of them, and
 *                      do not change their events while the batch exists
 *   seeds[P], streams[P]  resample keys of each problem (Philox key as in
 *                      hawkes_resample_locations), or both NULL for no resample
 *   flags              HAWKES_F32, optionally | HAWKES_MODEL1 | HAWKES_SKIP_UNDERFLOW
 *                      | HAWKES_BG_TIME
 *   cuda_stream        stream for the batch's work, or NULL for its own
 */
typedef struct hawkes_batch hawkes_batch;
int hawkes_batch_create(hawkes_batch** out, hawkes_ctx* const* problems, int32_t n_problems,
                        const uint64_t* seeds, const uint64_t* streams, uint32_t flags,
                        void* cuda_stream);
void hawkes_batch_destroy(hawkes_batch* batch);

/*
 * Queue one batched evaluation at resample iteration `iteration`.
 *   d_params  device pointer to P hawkes_params (problem p uses d_params[p])
 *   d_out     device pointer to 7 P doubles (problem p writes d_out[7p .. 7p+6])
 * If the batch was captured with these same two pointers, the captured CUDA
 * graph is launched; otherwise the kernels are queued one by one.  Returns
 * without waiting; see hawkes_batch_wait.
 */
int hawkes_batch_run(hawkes_batch* batch, const hawkes_params* d_params, uint64_t iteration,
                     double* d_out);

/*
 * Capture the whole evaluation (resample, staging, the single sweep launch,
 * per-problem reductions) into a CUDA graph bound to d_params and d_out; later
 * hawkes_batch_run calls with the same pointers replay it.  The iteration is
 * read from device memory written just before each launch.
 */
int hawkes_batch_capture(hawkes_batch* batch, const hawkes_params* d_params, double* d_out);

/* Wait for the batch's queued work; return the first latched device error. */
int hawkes_batch_wait(hawkes_batch* batch);

/*
 * Autotune the batch over the sweep variant, the column-chunk length of a
 * work item (16, 32 or 64 tiles of 256 sources), the item order (0: all
 * items longest first; 1: problem by problem, largest problem first, each
 * longest first) and the chains per CTA (1, 2 or 4; see
 * hawkes_batch_set_chains_per_cta).  Each configuration's sweep launches
 * are timed `reps` times with CUDA events after a warm-up, at d_params /
 * d_out (device pointers as for hawkes_batch_run); the fastest is kept.
 * Outputs (optional): the chosen variant, chunk length, order and mean sweep
 * time in ms (hawkes_batch_get_config also gives the chains per CTA).  Drops
 * a captured graph (capture again after tuning).
 */
int hawkes_batch_tune(hawkes_batch* batch, const hawkes_params* d_params, double* d_out, int reps,
                      int* variant, int* chunk, int* order, double* best_ms);

/* Select the sweep variant, chunk length and item order directly (drops a captured graph). */
int hawkes_batch_set_config(hawkes_batch* batch, int variant, int chunk, int order);

/*
 * Chains per CTA.  MCMC chains of one data set (Sec. 3.2 runs 30) share their
 * event times and differ in their location draws (Sec. 2.2) and parameters.
 * With chains_per_cta = k > 1, the problems of the batch whose event times
 * are identical (same n, bit-identical times; found when the batch is made)
 * are split, in batch order, into groups of k, and each group is swept by a
 * kernel whose CTAs take one row tile of the shared event order for all k
 * chains at once: one TMA copy stages the column tile of all k chains, and
 * each pair's time difference is formed once for the k chains.  Problems left
 * over (other event times, or the remainder of a class) are swept one per
 * item as with k = 1.  Results equal those of k = 1 up to FP32 rounding.
 *   chains_per_cta  1, 2 or 4; k > 1 only with the space-time background's
 *                   full gradient (not with HAWKES_BG_TIME, HAWKES_LOGLIK_ONLY
 *                   or HAWKES_SKIP_UNDERFLOW): HAWKES_ERR_ARG otherwise
 * Keeps the variant, chunk length and order; drops a captured graph.  The
 * group kernel's tile buffer (104 B per event and chain pair at k = 2) is
 * allocated here.
 */
int hawkes_batch_set_chains_per_cta(hawkes_batch* batch, int chains_per_cta);

/*
 * The batch's current configuration (outputs optional): sweep variant, chunk
 * length, item order, chains per CTA, and the number of groups swept with
 * several chains per CTA (0 when chains_per_cta is 1 or no k problems share
 * their times).
 */
int hawkes_batch_get_config(const hawkes_batch* batch, int* variant, int* chunk, int* order,
                            int* chains_per_cta, int* n_groups);

/*
 * As hawkes_batch_tune, through the autotuner cache (see hawkes_tune_cached
 * for the file and the key).  On a hit the cached configuration is selected
 * without timing (*from_cache = 1); on a miss the search runs and its result
 * is stored.  Outputs (optional) as for hawkes_batch_tune, without the time.
 */
int hawkes_batch_tune_cached(hawkes_batch* batch, const hawkes_params* d_params, double* d_out,
                             int reps, const char* cache_path, int* variant, int* chunk,
                             int* order, int* from_cache);

/*
 * Surrogate network (no counterpart in the paper: the learned part layered on
 * its method).  A 7 -> 256 -> 256 -> 7 multilayer perceptron with tanh hidden
 * units maps (six standardised log-parameters, z) to the standardised
 * log-likelihood and its six log-parameter partials d ell / d log p_k, where
 * z is either the constant 1 or a standardised feature supplied with each
 * sample (e.g. a summary of the location draw the log-likelihood was
 * evaluated under, so that the network can follow the cut posterior's
 * draw-to-draw changes).
 * Trained on the GPU by this library's kernels (BF16 products on the
 * 5th-generation tensor cores with the FP32 accumulator in tensor memory for
 * the 256 x 256 layer, FP32 elsewhere, Adam), evaluated inside HMC leapfrog
 * trajectories; the exact kernel keeps the accept/reject step.  A bounded
 * device wait of the tensor-core kernels that gives up is latched and
 * returned (HAWKES_ERR_TIMEOUT) by the next hawkes_mlp_train,
 * hawkes_mlp_loss_grad or hawkes_mlp_wait.
 *
 * Parameters, flattened (HAWKES_MLP_NPARAMS floats): W1[256 x 7], b1[256],
 * W2[256 x 256], b2[256], W3[7 x 256], b3[7], row-major.
 */
#define HAWKES_MLP_NPARAMS 69639
typedef struct hawkes_mlp hawkes_mlp;

/* Create with Glorot-uniform weights (Philox stream `seed`) and zero biases. */
int hawkes_mlp_create(hawkes_mlp** out, int device, void* cuda_stream, uint64_t seed);
void hawkes_mlp_destroy(hawkes_mlp* mlp);
int hawkes_mlp_get_params(hawkes_mlp* mlp, float* params);        /* host [NPARAMS], synchronous */
int hawkes_mlp_set_params(hawkes_mlp* mlp, const float* params);  /* also resets the Adam state */

/*
 * Training set: X[n x 6] log-parameters, F[n] the feature of each sample (or
 * NULL: the seventh input is the constant 1) and Y[n x 7] (log-likelihood,
 * six log-parameter partials), host arrays, n >= 2.  Column means and
 * standard deviations are computed on the device; inputs, feature and
 * targets are standardised with them (and predictions are mapped back).
 */
int hawkes_mlp_set_data(hawkes_mlp* mlp, int64_t n, const double* X, const double* F,
                        const double* Y);

/*
 * `steps` Adam steps (learning rate lr, betas 0.9 / 0.999) on minibatches of
 * `batch` rows (a multiple of 64, at most 4096) drawn with replacement by a
 * Philox stream keyed by `seed` and the step count.  *last_loss (optional)
 * receives the last minibatch's mean squared error (standardised units).
 */
int hawkes_mlp_train(hawkes_mlp* mlp, int64_t steps, int batch, double lr, uint64_t seed,
                     double* last_loss);

/*
 * One forward and backward pass without an update, for testing: host inputs
 * Xs[batch x 7] and targets Ts[batch x 7] in standardised units; outputs the
 * loss, the gradient grad[NPARAMS] and the network outputs Y[batch x 7]
 * (optional pointers).
 */
int hawkes_mlp_loss_grad(hawkes_mlp* mlp, int batch, const float* Xs, const float* Ts,
                         double* loss, float* grad, float* Y);

/*
 * Predictions for `count` (1..4096) parameter vectors: d_logp[count x 6]
 * device log-parameters and d_feature[count] their features (device; NULL
 * exactly when the training set had none, else HAWKES_ERR_STATE) ->
 * d_out[count x 7] device (log-likelihood, six log-parameter partials),
 * queued on the network's stream.
 */
int hawkes_mlp_predict(hawkes_mlp* mlp, int64_t count, const double* d_logp,
                       const double* d_feature, double* d_out);

/*
 * Standardisation statistics (host, 28 doubles): mean_in[6], sd_in[6],
 * mean_out[7], sd_out[7], then the feature's mean and sd (0 and 1 without a
 * feature).
 */
int hawkes_mlp_stats(hawkes_mlp* mlp, double* stats28);

/* Wait for the network's queued work. */
int hawkes_mlp_wait(hawkes_mlp* mlp);

/* Number of events n of the current set (0 if none). */
int64_t hawkes_num_events(const hawkes_ctx* ctx);

/*
 * Failure-detection self-check (synchronous).  Device-side waits (on the
 * sweep's TMA barriers) are bounded: after about 2 s a wait gives up, latches
 * HAWKES_ERR_TIMEOUT and the kernel returns, leaving the context usable.
 * This launches one thread that waits on a barrier nothing completes and
 * returns HAWKES_OK if that wait gave up and reported HAWKES_ERR_TIMEOUT as
 * designed (*seconds, optional: how long it took), an error otherwise.
 */
int hawkes_check_bounded_wait(hawkes_ctx* ctx, double* seconds);

/*
 * Debug build.  Compiled with -DHAWKES_DEBUG (lib/libhawkes_debug.so), the
 * kernels check every index they derive from a work list or a fix-up list
 * before using it: a work item must lie inside its problem's causal
 * triangle and padded arrays, a batch item's problem index must exist, and
 * a fix-up row must be an event.  A failed check skips the access and
 * latches HAWKES_ERR_BOUNDS, returned by the next synchronous call.  This is
 * the library's own stand-in for a memory checker; release builds compile
 * the checks out.
 *
 * hawkes_debug_build: 1 in the debug build, 0 otherwise.
 * hawkes_debug_set_item: debug build only (else HAWKES_ERR_STATE): overwrite
 *   work item k of the context's symmetric work list with (row tile,
 *   first column tile, end column tile), to exercise the checks.  A test
 *   hook; evaluations use the altered list until the next
 *   hawkes_set_events or hawkes_set_sweep_variant rebuilds it.
 */
/*
 * Events per time window of the HAWKES_SKIP_SPATIAL order (>= 256; default
 * 131,072).  Longer windows make tiles more compact in space and skip more
 * pairs, at the cost of a wider time span per tile (times are carried in two
 * FP32 words, so precision holds).  At N = 1,000,000 over 1,200 days the
 * sweep took 99, 65, 47, 38 and 41 ms with windows of 16k, 32k, 64k, 128k
 * and 256k events.  Takes effect at the next evaluation with the flag.
 */
int hawkes_set_spatial_window(hawkes_ctx* ctx, int64_t events);

int hawkes_debug_build(void);
int hawkes_debug_set_item(hawkes_ctx* ctx, int k, int row_tile, int col_begin, int col_end);

/*
 * Allocation-free log-likelihood and gradient (no counterpart in the paper;
 * a deployment convenience of this library).
 *
 * For callers that cannot allocate device memory: code running inside a
 * custom device allocator or memory-pool callback (a cudaMalloc there would
 * recurse into the allocator), applications that reserve all device memory
 * up front and account for every byte, and threads that must not block on
 * the allocator's device-wide synchronisation.  This call allocates and frees
 * nothing, on the device or through any library.  Its scratch space is one
 * fixed array built into the library (about 10 MB), which every GPU that
 * loads the library holds until the process exits.
 *
 *   d_t[n]        device pointer: event times, > 0, non-decreasing
 *   d_x[n], d_y[n] device pointers: event locations
 *   d_s[n]        device pointer: per-event source bandwidth scale s_j > 0
 *                 (eq. 3), or NULL for s_j = 1 (eq. 2)
 *   n             1 <= n <= HAWKES_NOALLOC_MAX_N (65,536); larger n returns
 *                 HAWKES_ERR_TOO_LARGE
 *   d_params      device pointer to one hawkes_params
 *   flags         HAWKES_F32, optionally | HAWKES_MODEL1 | HAWKES_BG_TIME (the
 *                 FP64 path and tile skipping are not offered here)
 *   d_out         device pointer to 7 doubles: ell, then the six partials
 *   cuda_stream   cudaStream_t of the current device to queue the work on
 *                 (NULL: the legacy default stream)
 * Computes the same quantity as hawkes_loglik_grad (whole sum, FP32 pair
 * terms) on the current CUDA device and returns without waiting.  Invalid
 * events detected on the device (unsorted or non-positive times, non-finite
 * values) make all 7 outputs NaN.  The first call on each device looks up the
 * scratch array's device address and sets kernel attributes; make that first
 * call before any stream capture.  All calls on a device share the scratch
 * array, which keeps the previous call's contents (each call clears what must
 * start at zero): calls whose work can overlap on the GPU, e.g. on two
 * streams, race and must be serialised by the caller.
 */
#define HAWKES_NOALLOC_MAX_N 65536
int hawkes_loglik_grad_noalloc(const double* d_t, const double* d_x, const double* d_y,
                               const double* d_s, int64_t n, const hawkes_params* d_params,
                               uint32_t flags, double* d_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HAWKES_H */
