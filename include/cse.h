/*
 * cse.h -- C ABI of the GB300 Continuous Simulation Extension (CSE) hot path.
 *
 * Method: Yang, Thompson & Sklar, "Guarantees for Comprehensive Simulation
 * Assessment of Statistical Methods" (arXiv 2212.10042).  CSE simulates a trial
 * design at the simulation point theta_i of every tile H_i of a platten
 * (Def. tile/platten), then extends each point estimate to the whole tile with
 * the Tilt-Bound (Thm. tilt-bound), either as a confidence bound on the Type I
 * Error (Validation, Alg. validation) or as a calibrated rejection threshold
 * (Calibration, Alg. calibration).
 *
 * Conventions shared by every call:
 *   - Data model: d independent Bernoulli arms on the logit scale, embedded in
 *     the i.i.d. model with n_max patients per arm (Sec. 9, adaptive embedding
 *     of binomial arms): A(theta) = sum_a n_max log(1 + e^theta_a),
 *     T_a(X) = successes of arm a over all n_max patients.
 *   - Common random numbers (Sec. 7.3): uniform word j of sim k, arm a is word
 *     j mod 4 of Philox4x32-10(counter = (k, a, j/4, 0), key = seed); every tile
 *     uses the same sims; a tile with K_i sims uses sims 0..K_i-1.  Patient j
 *     succeeds iff u < floor(2^32 sigmoid(theta_a)) (FP64).
 *   - A design rejects iff S(X) < lambda (Sec. 7, f_lambda = P(S < lambda)).
 *   - All array arguments are DEVICE pointers unless marked "host".  Output
 *     buffers are caller-owned; scratch (uniforms, count tables, work queues)
 *     is owned by the context.  Calls are asynchronous on `stream` unless said
 *     otherwise.  A context is not thread-safe; use one per host thread.
 *   - Every call returns a cse_status; nothing throws across the ABI.
 */
#ifndef CSE_H_
#define CSE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* cse_stream_t;
typedef struct cse_ctx cse_ctx;

typedef enum {
    CSE_OK = 0,
    CSE_INVALID_ARG = -1,        /* a documented argument range was violated */
    CSE_UNSUPPORTED_DESIGN = -2, /* design outside the supported statistics / sizes */
    CSE_OOM = -3,                /* device allocation of context scratch failed */
    CSE_CUDA_ERROR = -4,         /* a CUDA runtime call or kernel launch failed */
    CSE_DEVICE_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    CSE_DEVICE_CHECK = -6,       /* a device-side argument check failed (e.g. K_i > K_max) */
    CSE_CAPACITY = -7            /* request larger than the fixed scratch of cse_simulate_tiles_static */
} cse_status;

typedef enum {
    CSE_STAT_ONE_ARM_Z = 0,        /* S = -(x - n p0)/sqrt(n p0 (1-p0)), FP32 */
    CSE_STAT_TWO_ARM_POOLED_Z = 1, /* S = -(p1 - p0)/sqrt(pbar(1-pbar)(1/n0+1/n1)), FP32 */
    CSE_STAT_BAYES4 = 2,           /* four-arm hierarchical selection design, FP32 posterior */
    CSE_STAT_BERRY4 = 3            /* four-arm basket trial (Sec. 10.1), one analysis, FP32 posterior:
                                      S = min over the tile's null arms of 1 - P(theta_i > t_i | x),
                                      reject iff S < lambda (lambda = 0.15 is the 85% rule) */
} cse_stat_id;

/* Trial design (host struct, copied by cse_create). */
typedef struct {
    int32_t stat;       /* cse_stat_id */
    int32_t d;          /* arms: 1 for ONE_ARM_Z, 2 for TWO_ARM_POOLED_Z, 4 for BAYES4 and BERRY4 */
    int32_t n_looks;    /* analyses, 1..3 (only BAYES4 uses more than one) */
    int32_t look_n[3];  /* cumulative patients per arm at each analysis; look_n[n_looks-1]
                           is n_max, 1 <= n_max <= 128 */
    double p0;          /* ONE_ARM_Z null proportion (0.5) */
    double drop;        /* BAYES4 interim drop threshold on P(theta_i > theta_0 | data) (0.1) */
    double arm_null[4]; /* BERRY4: t_i, the logit of arm i's null response rate; the model's
                           offset log-odds are logit(p_i) - t_i and H_i is theta_i <= t_i.
                           BERRY4 requires n_looks = 1 and n_max <= 63 (the posterior table
                           holds (n_max + 1)^4 states of 16 bytes).  Ignored otherwise. */
} cse_design;

/*
 * Tile set in axis-indexed form (Def. tile/platten).  Tile i is the box
 * [c_i - h_i, c_i + h_i] with simulation point c_i, where
 * c_i[a] = axis[a][center_idx[i*d + a]].  axis[a] holds the distinct centre
 * coordinates of arm a (any order).  null_mask[i] bit j-1 is set when the
 * tile's box meets null hypothesis H_j (theta_j <= theta_0; one-arm:
 * theta <= 0; BERRY4: bit j for H_j = {theta_j <= t_j}, j = 0..3); the FWER
 * indicator then counts rejections of those hypotheses only (Sec. 5, F_b).
 * All pointers are device pointers.  A tile must have null_mask[i] != 0 and
 * half-widths h >= 0 (h = 0: a point); the bound and calibration passes check
 * this on the device, give such a tile NaN bounds (alpha' NaN, lambda_i -inf)
 * and record a DEVICE_CHECK error that cse_sync reports.
 */
typedef struct {
    int64_t n_tiles;
    int32_t n_axis[4];          /* host: entries of axis[a] */
    const double* axis[4];      /* device [n_axis[a]] */
    const int32_t* center_idx;  /* device [n_tiles * d] */
    const double* halfwidth;    /* device [n_tiles * d], >= 0 (0: a point) */
    const uint32_t* null_mask;  /* device [n_tiles], != 0 */
    const int32_t* K;           /* device [n_tiles], 1 <= K_i <= K_max of the set */
    int32_t K_max;              /* host: max_i K_i (<= the context's K_max) */
} cse_tiles;

/* Context: copies the design, generates the CRN uniforms for sims
 * 0..K_max-1 (Philox4x32-10, key = seed), sorts them within each
 * (sim, arm, analysis segment), and builds the statistic tables.  Owns all
 * scratch.  Synchronises `stream` before returning.
 * Errors: INVALID_ARG (null out, K_max < 1 or > 1<<20), UNSUPPORTED_DESIGN,
 * OOM, CUDA_ERROR. */
int cse_create(cse_ctx** out, const cse_design* design, uint64_t seed, int32_t K_max,
               cse_stream_t stream);

/* Frees the context and its scratch (synchronises the device first). NULL is OK. */
int cse_destroy(cse_ctx* ctx);

/*
 * Simulation at every tile's point (Sec. 6.1, input of Alg. validation step 2):
 *   R_out[i]          = sum_{k<K_i} 1{S_ik < lambda}                 (int64)
 *   Xrej_out[i*d+a]   = sum_k 1{S_ik < lambda} T_a(X_ik)              (int64)
 *   score_out[i*d+a]  = Xrej - n_max sigmoid(c_i[a]) R   (score-function sum
 *                       sum_k 1{rej}(T - grad A(theta)), Ex. exp-fam) (double)
 * Any output pointer may be NULL.  Errors: INVALID_ARG, DEVICE_CHECK (a tile
 * with K_i outside [1, K_max]; reported by the next call or cse_sync), CUDA_ERROR.
 */
int cse_simulate_tiles(cse_ctx* ctx, const cse_tiles* tiles, double lambda,
                       int64_t* R_out, int64_t* Xrej_out, double* score_out,
                       cse_stream_t stream);

/*
 * Monte Carlo Type I Error at arbitrary points (Sec. 6.1; Ex. exp-fam for the
 * score), with the points given by their coordinates instead of an
 * axis-indexed tile set:
 *   fhat_out[i]      = R_i / K_i, the estimate of f(theta_i)          (double)
 *   R_out, Xrej_out, score_out as in cse_simulate_tiles (each may be NULL)
 * theta: device [n_points * d] (point i's coordinate of arm a at i*d + a);
 * null_mask: device [n_points] (the hypotheses the FWER statistic counts, as in
 * cse_tiles); K: device [n_points], 1 <= K_i <= K_max; K_max (host) <= the
 * context's.  The library gathers each arm's distinct coordinates on the device
 * (equal bit patterns share one simulation; every NaN is one coordinate) and
 * then runs the simulation of cse_simulate_tiles.  Synchronises `stream` once,
 * after the gathering, to size the count tables.  Scratch grows with n_points
 * and is owned by the context.  Errors: INVALID_ARG (NULL context, theta,
 * null_mask, K or fhat_out; n_points < 1 or > 2^28; K_max outside
 * [1, the context's]), OOM, CUDA_ERROR, DEVICE_CHECK (a point with K_i outside
 * [1, K_max]; reported by the next call or cse_sync).
 */
int cse_type1_error(cse_ctx* ctx, int64_t n_points, const double* theta, const uint32_t* null_mask,
                    const int32_t* K, int32_t K_max, double lambda, double* fhat_out,
                    int64_t* R_out, int64_t* Xrej_out, double* score_out, cse_stream_t stream);

/*
 * Validation (Alg. validation) at threshold lambda with confidence 1 - delta:
 *   u0_out[i]    = Clopper-Pearson upper bound Beta^-1(1-delta; R+1, K-R)
 *                  (Eq. clopper-pearson:def; 1 when R = K)
 *   bound_out[i] = inf_{q>=1} max_{v in vertices} U(c_i, v, q, u0)
 *                  (Eq. tilt-bound:exp-fam, Eq. optimized-tilt-bound-tile; Thm. 3
 *                  reduces the sup over the box to its 2^d vertices)
 *   qstar_out[i] = the minimising q (+inf for the q -> inf limit)
 * R/Xrej/score outputs as in cse_simulate_tiles (each may be NULL).
 * Errors: INVALID_ARG (delta not in (0,1)), as cse_simulate_tiles.
 */
int cse_validate(cse_ctx* ctx, const cse_tiles* tiles, double lambda, double delta,
                 int64_t* R_out, int64_t* Xrej_out, double* score_out,
                 double* u0_out, double* bound_out, double* qstar_out, cse_stream_t stream);

/*
 * Lower validation bound (Rem. extension-lower: the Tilt-Bound applied to
 * 1 - F bounds f from below) at threshold lambda with confidence 1 - delta:
 *   l0_out[i]    = lower Clopper-Pearson bound Beta^-1(delta; R, K-R+1), the l
 *                  with P(Binom(K, l) >= R) = delta (0 when R = 0)
 *   lower_out[i] = 1 - inf_{q>=1} max_{v in vertices} U(c_i, v, q, 1 - l0): for
 *                  every theta in the box f(theta) >= lower_out[i] with
 *                  probability >= 1 - delta (0 when uninformative)
 *   qstar_out[i] = the minimising q of the inner bound
 * R/Xrej/score outputs as in cse_simulate_tiles (each may be NULL).
 * Errors: INVALID_ARG (delta not in (0,1)), as cse_simulate_tiles.
 */
int cse_validate_lower(cse_ctx* ctx, const cse_tiles* tiles, double lambda, double delta,
                       int64_t* R_out, int64_t* Xrej_out, double* score_out,
                       double* l0_out, double* lower_out, double* qstar_out,
                       cse_stream_t stream);

/*
 * Two-sided validation band: one simulation pass, then the lower bound of
 * cse_validate_lower and the upper bound of cse_validate, each at delta / 2,
 * so that lower_out[i] <= f(theta) <= upper_out[i] for every theta in box i
 * holds with probability >= 1 - delta (union bound).  l0/u0 are the two
 * Clopper-Pearson bounds at delta / 2.  Any output pointer may be NULL.
 * Errors: INVALID_ARG (delta not in (0,1)), as cse_simulate_tiles.
 */
int cse_validate_band(cse_ctx* ctx, const cse_tiles* tiles, double lambda, double delta,
                      int64_t* R_out, int64_t* Xrej_out, double* score_out,
                      double* l0_out, double* lower_out, double* u0_out, double* upper_out,
                      cse_stream_t stream);

/*
 * Calibration (Alg. calibration) at level alpha:
 *   alpha_prime_out[i] = sup_q min_v U^-1(c_i, v, q, alpha)   (Eq. tilt-bound-inv,
 *                        Eq. tile-calibration-final)
 *   lambda_tile_out[i] = S_(k_i) among S_i1..S_iK_i, k_i = floor((K_i+1) alpha'_i)
 *                        (Eq. calibrated-threshold; -inf when k_i = 0)
 *   *lambda_out (HOST) = min_i lambda_tile (Eq. calibrated-threshold-final)
 * Synchronises `stream` to return lambda_out.  Errors: INVALID_ARG (alpha not in (0,1)).
 */
int cse_calibrate(cse_ctx* ctx, const cse_tiles* tiles, double alpha,
                  double* alpha_prime_out, double* lambda_tile_out, double* lambda_out,
                  cse_stream_t stream);

/*
 * Randomised test (Sec. 7, after Thm. calibration: an independent uniform w
 * adjoined to each sim removes the ties of a discrete statistic; statistic and
 * threshold become pairs compared lexicographically).  The one- and two-arm
 * z-test designs only (UNSUPPORTED_DESIGN otherwise).  Sim k's word is word 0
 * of Philox4x32-10(counter (k, 0, 0, 1), key = seed), regenerated with the
 * uniforms after cse_reseed.
 *
 * cse_validate_rand: as cse_validate with the rule "reject iff S < lambda, or
 * S = lambda and w < c" (c = 0: the plain rule S < lambda).
 */
int cse_validate_rand(cse_ctx* ctx, const cse_tiles* tiles, double lambda, uint32_t c, double delta,
                      int64_t* R_out, int64_t* Xrej_out, double* score_out,
                      double* u0_out, double* bound_out, double* qstar_out,
                      cse_stream_t stream);

/*
 * cse_calibrate_rand: as cse_calibrate with pairs: per tile the
 * k_i-th smallest pair (S, w) of its sims, k_i = floor((K_i + 1) alpha'_i)
 * (Eq. calibrated-threshold; (-inf, 0) when k_i = 0) in lambda_tile_out[i] and
 * c_tile_out[i] (both required, device), and the lexicographic minimum over
 * tiles (Eq. calibrated-threshold-final) in *lambda_out and *c_out (host, may be
 * NULL).  A tile's own sims then reject exactly k_i - 1 times at its pair.
 * Synchronises `stream`.  Errors: INVALID_ARG (alpha not in (0,1), a NULL
 * per-tile output), UNSUPPORTED_DESIGN, OOM, as cse_simulate_tiles.
 */
int cse_calibrate_rand(cse_ctx* ctx, const cse_tiles* tiles, double alpha,
                       double* alpha_prime_out, double* lambda_tile_out, uint32_t* c_tile_out,
                       double* lambda_out, uint32_t* c_out, cse_stream_t stream);

/*
 * One fused pass of the whole path: simulation at `lambda` (R, Xrej, score),
 * validation bounds at `delta`, and calibration at `alpha` (alpha', per-tile
 * lambda, global lambda written to the DEVICE scalar lambda_dev).  The per-sim
 * statistics are computed once and serve both the rejection counts and the
 * order statistics.  Asynchronous (no host sync).  Any per-tile output may be
 * NULL except lambda_tile_out and lambda_dev.
 */
int cse_step(cse_ctx* ctx, const cse_tiles* tiles, double lambda, double delta, double alpha,
             int64_t* R_out, int64_t* Xrej_out, double* score_out,
             double* u0_out, double* bound_out, double* qstar_out,
             double* alpha_prime_out, double* lambda_tile_out, double* lambda_dev,
             cse_stream_t stream);

/*
 * Backward of the Monte Carlo Type I Error f_hat_i = R_i / K_i with respect to
 * the tile point theta_i: grad_theta[i*d+a] = grad_out[i] * score[i*d+a] / K_i,
 * the score-function estimate of grad f = E[F (T - grad A)] (Ex. exp-fam).
 */
int cse_score_backward(int64_t n_tiles, int32_t d, const double* grad_out, const double* score,
                       const int32_t* K, double* grad_theta, cse_stream_t stream);

/* The statistic S of every simulated trial: S_out[offsets[i] + k] for sim k of
 * tile i (FP32, the value the design compares with lambda; +inf when the
 * four-arm design has no rejectable true-null arm).  offsets: device int64
 * [n_tiles], caller-owned, each range [offsets[i], offsets[i] + K_i) inside
 * S_out.  For testing and export; the other calls never store per-sim values. */
int cse_statistics(cse_ctx* ctx, const cse_tiles* tiles, const int64_t* offsets, float* S_out,
                   cse_stream_t stream);

/* Sets the key of the context's CRN uniforms to `seed` (a new batch of
 * simulations; same layout and sorting as cse_create).  No kernel runs here:
 * the next call that simulates regenerates the uniforms (and the randomised
 * test's words) on its own stream before its success counts, after it has
 * started its tile-only work (alpha', on the context's second stream), so the
 * two overlap.  `stream` is not used.  Errors: INVALID_ARG (NULL ctx). */
int cse_reseed(cse_ctx* ctx, uint64_t seed, cse_stream_t stream);

/* Autotuner: times the fused simulation pass of `tiles` (at `lambda`, with the
 * calibration selection for level `alpha`) in each configuration of the z-test
 * cell-histogram kernel, (threads per block, tiles per block) in (128, 1),
 * (256, 1), (512, 1), (64, 1), (128, 2), (256, 2), (256, 4) -- a block of T
 * threads working on G tiles at once gives each tile T / G threads, so the sims
 * per block and step are 16 T and the tiles in flight per SM follow from the
 * blocks that fit -- and keeps the fastest for this context's later calls (the
 * plain path: its per-sim kernel at 128, 256, 512 threads).  *threads_out and
 * *tiles_out (host, may be NULL) receive the choice.  The four-arm designs have
 * one configuration each: (512, 1) for the selection design's tabulated form
 * when its codes fit the packed per-trial form, else (256, 1).  Synchronises
 * `stream`.  Results never depend on
 * the choice.  Errors: INVALID_ARG, as cse_simulate_tiles. */
int cse_autotune(cse_ctx* ctx, const cse_tiles* tiles, double lambda, double alpha, int32_t* threads_out,
                 int32_t* tiles_out, cse_stream_t stream);

/* Options.  CSE_OPT_BAYES_DIRECT (BAYES4 and BERRY4 designs only): 1 evaluates the
 * FP32 posterior for every simulated trial; 0 (default when the count-state tables
 * fit, at most 2^27 entries) reads the posterior tabulated once per context over all
 * reachable success-count states.  Both evaluate the same FP32 function. */
enum { CSE_OPT_BAYES_DIRECT = 1, CSE_OPT_PLAIN = 2, CSE_OPT_SIM_THREADS = 3, CSE_OPT_CELLS_BOX = 4,
       CSE_OPT_PDL = 5, CSE_OPT_SIM_TILES = 7 };
/* CSE_OPT_PLAIN: 1 selects the plain comparison path with the same results:
 * success counts by one binary search per (tile, sim, arm) in the sorted
 * uniforms (no axis count table), the bound pass entirely in FP64 (bisection
 * over q, Newton for Clopper-Pearson, no FP32 stage), and for BAYES4 and BERRY4
 * the direct per-trial posterior.  0 (default) is the chosen path.
 * CSE_OPT_SIM_THREADS (z-test designs): 64, 128, 256 or 512 fixes the block size
 * of the simulation kernels with one tile per block (64: the cell kernel only;
 * default 128).  CSE_OPT_SIM_TILES (z-test designs): 1, 2 or 4 tiles per block of
 * the cell kernel at the current block size, where that configuration is built
 * (see cse_autotune).
 * CSE_OPT_CELLS_BOX (z-test designs): the number of cells of a tile's box of
 * reachable count cells that the simulation kernel histograms at once (0, the
 * default: min(4096, count table) for tiles of 128 or more threads, 2048 for
 * smaller ones); a larger box is done in slabs of whole rows, one pass over the
 * sims per slab.  Same results at any value; a value from the longest row
 * (n_max + 1 for the two-arm design, 1 for one arm) up to min(2048, count table)
 * exercises the slab path.
 * CSE_OPT_PDL: 1 launches the kernels that run one after another in the
 * caller's stream (uniforms, count tables, the z-test simulation,
 * Clopper-Pearson, bounds, minimum) with programmatic dependent launch: each
 * may be scheduled while the one before it finishes and waits for it before
 * touching memory.  0 (default) launches them in plain stream order.  Same
 * results.  It pays where launch latency dominates (one arm, 64 tiles: 0.142
 * -> 0.133 ms per step) and costs time on large batches (two-arm 256²: 0.626
 * -> 0.638 ms per step).
 * Errors: INVALID_ARG (unknown option or value, or an option of the other
 * design family), UNSUPPORTED_DESIGN (BAYES_DIRECT = 0 without the tables). */
int cse_set_option(cse_ctx* ctx, int option, int64_t value);

/* Per-kernel timing: when enabled, every kernel this context launches is
 * bracketed by CUDA events recorded on its launch stream.  cse_profile_read
 * synchronises the device, then fills up to `max` entries with the kernel
 * name, its number of launches and their summed duration in milliseconds, and
 * returns the number of entries (or a negative status).  Reading resets. */
int cse_profile_enable(cse_ctx* ctx, int enable);
int cse_profile_read(cse_ctx* ctx, const char** names, int64_t* launches, double* total_ms, int max);

/* Restricts the per-kernel timing to one kernel group, `name` being one of the
 * names cse_profile_read reports (e.g. "sim_ztest"); NULL or "" times every
 * group again.  The other kernels then run without events around them (each
 * pair costs a few microseconds of step time and can delay a kernel on another
 * stream).  Errors: INVALID_ARG (null context or an unknown name). */
int cse_profile_only(cse_ctx* ctx, const char* name);

/*
 * Allocation-free simulation (the paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory, e.g. a plugin in a
 * host program that owns all GPU memory, or code that must not risk the device
 * synchronisation cudaMalloc/cudaFree can cause).  Same outputs as
 * cse_create(design, seed, tiles->K_max) followed by cse_simulate_tiles, for
 * the one- and two-arm z-test designs, but every scratch buffer lives in one
 * fixed 32 MiB array of device global memory inside this library (held by
 * every GPU that loads it until the process exits); nothing is allocated.
 * Capacity: 256 + 4 d K_max n_max + 20 NA + NA ceil16(K_max) + 10 (n_max+1)^d
 * bytes (NA = sum of n_axis, each term rounded up to 256) must fit in 32 MiB
 * (e.g. two arms, n_max = 100, K_max = 16384, NA = 512: ~21.6 MB, 20.6 MiB);
 * larger requests return CSE_CAPACITY before any GPU work.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current.  The call cannot be captured into a CUDA graph: it reads the
 * device-side error flag back and synchronises `stream`, so on a stream that is
 * capturing it returns CSE_INVALID_ARG without touching the capture.  All calls share the
 * array, which keeps the previous call's contents (the call clears its flags
 * itself); calls whose GPU work overlaps (other streams, other host threads)
 * race on it and must be serialised by the caller.  Synchronises `stream`
 * before returning so that device-side checks are reported (DEVICE_CHECK).
 * Errors: INVALID_ARG (also: `stream` is capturing), UNSUPPORTED_DESIGN (not a
 * z-test design), CAPACITY,
 * DEVICE_CHECK, CUDA_ERROR.
 */
int cse_simulate_tiles_static(const cse_design* design, uint64_t seed, const cse_tiles* tiles,
                              double lambda, int64_t* R_out, int64_t* Xrej_out, double* score_out,
                              cse_stream_t stream);

/*
 * Measured peak of one execution pipe (measurement support; the paper has no
 * counterpart).  Launches blocks_per_sm x (SM count) blocks of 256 threads, each
 * thread running `iters` iterations of 128 independent instructions of one kind,
 * once to warm up and then `reps` times between two CUDA events on `stream`:
 *   CSE_PROBE_ALU          lop3.b32 (3-input logic: the integer ALU pipe)
 *   CSE_PROBE_FMA          fma.rn.f32 (FP32 FMA pipe)
 *   CSE_PROBE_DFMA         fma.rn.f64 (FP64 pipe)
 *   CSE_PROBE_SMEM_ATOMIC  atom.shared.add.u32, each lane of a warp on its own
 *                          bank (conflict-free shared-memory atomics)
 * *ops_per_s (host, may be NULL) receives lane-operations per second (one warp
 * instruction = 32 lane-ops), *ms_per_launch (host, may be NULL) the mean
 * launch time.  Allocates and frees a 64-byte result word; synchronises
 * `stream`.  Errors: INVALID_ARG (unknown kind, blocks_per_sm outside 1..8,
 * iters outside 1..2^20, reps outside 1..1000), OOM, CUDA_ERROR, DEVICE_CHECK
 * (an atomic increment was lost).
 */
enum { CSE_PROBE_ALU = 0, CSE_PROBE_FMA = 1, CSE_PROBE_DFMA = 2, CSE_PROBE_SMEM_ATOMIC = 3 };
int cse_probe_peak(int kind, int32_t blocks_per_sm, int32_t iters, int32_t reps, double* ops_per_s,
                   double* ms_per_launch, cse_stream_t stream);

/* Blocks until `stream` is idle, then reports (and clears) any device-side
 * check or timeout recorded by earlier calls of this context. */
int cse_sync(cse_ctx* ctx, cse_stream_t stream);

/* Static description of a status code. */
const char* cse_status_str(int status);

/* Number of this library's kernels launched by the calling context so far. */
int64_t cse_launch_count(const cse_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CSE_H_ */
