/*
 * gmq.h -- C ABI of the GB300 adaptive Genz-Malik quadrature library.
 *
 * The library integrates f over a d-dimensional hyper-rectangle
 * Omega = [lo_1,hi_1] x ... x [lo_d,hi_d] to a relative/absolute tolerance
 * and returns the integral, its error estimate, and region and evaluation
 * counts (problem statement: paper Sec. 2, first display; stopping rule
 * eps <= max(abs_tol, rel_tol |I|): paper Sec. 4).  Every refinement sweep
 * runs on one GPU over a device-resident structure-of-arrays list of regions
 * (paper Sec. 3):
 *   1. the Genz-Malik degree-7 rule with its embedded degree-5 rule on every
 *      region, giving I_r, eps_r = |I7_r - I5_r| and the split axis from
 *      per-axis fourth differences (paper Sec. 2);
 *   2. the global sums I, eps and the convergence test (paper Sec. 3, 4);
 *   3. the classifier that retires regions with negligible error into
 *      running sums, with round-off guards (paper Sec. 3);
 *   4. bisection of the surviving regions along their axis through a
 *      scan-based compaction (paper Sec. 3, fused filter + split).
 *
 * Conventions for every call:
 *   - Every call returns a gmq_status and never throws or aborts.
 *   - Host pointers (gmq_problem arrays, gmq_options, gmq_result, seed
 *     outputs) are read or written during the call only; the caller keeps
 *     ownership.
 *   - Pointers named d_* are device pointers in the context's device memory
 *     (for example from torch.empty(..., device="cuda")); they are read or
 *     written on the context stream and the call waits for that work before
 *     returning, unless stated otherwise.
 *   - Region arrays are structure-of-arrays with leading dimension ld:
 *     centre k of region r is d_center[k*ld + r], half-width d_halfw[k*ld + r],
 *     0 <= k < dim, 0 <= r < n, ld >= n.
 *   - Calls on one context are not thread-safe; use one context per thread.
 */
#ifndef GMQ_H
#define GMQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Largest supported dimension. */
#define GMQ_MAX_DIM 16

typedef enum gmq_status {
  GMQ_OK = 0,              /* converged: error <= max(abs_tol, rel_tol |I|)   */
  GMQ_CAP_REACHED = 1,     /* next sweep would exceed max_regions; best estimate returned */
  GMQ_MAX_ITERS = 2,       /* max_iters sweeps done; best estimate returned   */
  GMQ_ROUNDOFF_LIMIT = 3,  /* every region retired (round-off guards) before the
                              tolerance was met; best estimate returned        */
  GMQ_ERR_INVALID = -1,    /* bad argument                                    */
  GMQ_ERR_OOM = -2,        /* device memory (or the caller's pool) too small  */
  GMQ_ERR_CUDA = -3,       /* a CUDA call failed                              */
  GMQ_ERR_NONFINITE = -4,  /* the integrand produced a NaN or an infinity     */
  GMQ_ERR_TIMEOUT = -5,    /* a bounded device wait gave up                   */
  GMQ_ERR_TOO_LARGE = -6   /* input longer than a fixed-size scratch allows   */
} gmq_status;

/* Built-in integrands (paper Sec. 4 test functions; Genz families).
 * a and u are per-axis parameters of length dim. */
typedef enum gmq_family {
  GMQ_OSCILLATORY = 0,   /* cos(2 pi u_1 + sum_j a_j x_j)                 */
  GMQ_PRODUCT_PEAK = 1,  /* prod_j 1 / (a_j^-2 + (x_j - u_j)^2)           */
  GMQ_CORNER_PEAK = 2,   /* (1 + sum_j a_j x_j)^-(dim+1)                  */
  GMQ_GAUSSIAN = 3,      /* exp(-sum_j a_j^2 (x_j - u_j)^2)               */
  GMQ_C0 = 4,            /* exp(-sum_j a_j |x_j - u_j|)                   */
  GMQ_DISCONTINUOUS = 5, /* 0 if any x_j > u_j, else exp(sum_j a_j x_j)   */
  GMQ_POLY_SUMSQ11 = 6,  /* (sum_j x_j^2)^11 (a, u unused)                */
  GMQ_NUM_FAMILIES = 7
} gmq_family;

typedef enum gmq_precision {
  GMQ_FP64 = 0,  /* every step in FP64                                       */
  GMQ_MIXED = 1  /* integrand in FP32 with compensated (two-sum) class sums;
                    error difference, axis choice and global sums in FP64   */
} gmq_precision;

typedef enum gmq_classifier {
  GMQ_VOLUME_SHARE = 0, /* retire r if eps_r <= max(abs_tol, rel_tol |I|) * vol_r / vol(Omega) */
  GMQ_LOCAL_REL = 1     /* retire r if eps_r <= rel_tol |I_r|                                    */
} gmq_classifier;

/* Quadrature rule (paper Sec. 3: the method is not tied to one rule).
 * GMQ_RULE_GENZ_MALIK: the degree-7 Genz-Malik rule with its embedded
 * degree-5 rule (Sec. 2), any dim.  GMQ_RULE_GAUSS_KRONROD: the
 * tensor-product Gauss-Kronrod rule, 7-point Gauss / 15-point Kronrod per
 * axis (15^dim nodes per region; the paper names the rule but not its order
 * -- this is the classic pair), FP64 only, dim <= GMQ_GK_MAX_DIM (Sec. 4
 * reports its cost as too high from dim 7 on).  Its error estimate is
 * |I_K - I_G|; its split axis is the one with the largest directional
 * estimate prod h_k |sum (prod_{j != k} wK)(wK_k - wG_k) f| (G7 along that
 * axis only), or the widest axis when all of those are below 1e-11 of the
 * terms' magnitude. */
typedef enum gmq_rule {
  GMQ_RULE_GENZ_MALIK = 0,
  GMQ_RULE_GAUSS_KRONROD = 1
} gmq_rule;

#define GMQ_GK_MAX_DIM 6

/* Local error estimate of the Genz-Malik rule (paper Sec. 2 names the
 * heuristic of Berntsen, Espelid & Genz 1991 without printing it).
 * GMQ_EST_EMBEDDED: eps_r = |I7_r - I5_r|, the difference of the degree-7
 * rule and its embedded degree-5 rule.  GMQ_EST_NULL_RULES: four fully
 * symmetric null rules on the same nodes (weight sums zero; degrees 5, 3,
 * 3 and 1; mutually orthogonal, each with the norm of the degree-7
 * weights), evaluated from the five class sums the rule already forms:
 * e1 = |N1|, e2 = sqrt(N2^2 + N3^2), e3 = |N4|, r = max(e1/e2, e2/e3) (x/0 =
 * infinity for x > 0, 0/0 = 0); eps_r = 10 max(e1, e2, e3) if r >= 1 (not
 * yet asymptotic), else 10 r e1 (e1 extrapolated by one observed decay
 * step: the degree-5 null rule is one step below the degree-7 rule).  The
 * form and constants are this library's reading of the heuristic; the node
 * work is the same, only the per-region epilogue changes. */
typedef enum gmq_estimator {
  GMQ_EST_EMBEDDED = 0,
  GMQ_EST_NULL_RULES = 1
} gmq_estimator;

typedef struct gmq_problem {
  int32_t dim;       /* 1 <= dim <= GMQ_MAX_DIM                             */
  int32_t family;    /* gmq_family                                          */
  const double *lo;  /* host, length dim; NULL means all zeros              */
  const double *hi;  /* host, length dim; NULL means all ones; hi > lo      */
  const double *a;   /* host, length dim (may be NULL for POLY_SUMSQ11)     */
  const double *u;   /* host, length dim (may be NULL for POLY_SUMSQ11)     */
} gmq_problem;

typedef struct gmq_options {
  double rel_tol;      /* relative tolerance tau_rel >= 0                   */
  double abs_tol;      /* absolute floor (paper: 1e-16)                     */
  int64_t max_regions; /* region cap per sweep; sizes the region pool       */
  int32_t init_splits; /* s: the initial partition has s^dim boxes;
                          0 = largest s with s^dim <= min(4096, max_regions) */
  int32_t max_iters;   /* sweep limit; 0 = 1000                             */
  int32_t precision;   /* gmq_precision                                     */
  int32_t classifier;  /* gmq_classifier                                    */
  int32_t lanes;       /* threads per region in the rule kernel: 0 = chosen
                          per sweep by the library, else 1, 4, 32 or (FP64
                          only) 128.  FP64 results do not depend on it
                          (every class sum is one fixed tree); mixed-
                          precision results do, at FP32 rounding level      */
  int32_t flags;       /* 0, or GMQ_KEEP_PARTITION                           */
  int32_t rule;        /* gmq_rule (GMQ_RULE_GENZ_MALIK by default)          */
  int32_t estimator;   /* gmq_estimator (GMQ_EST_EMBEDDED by default; the
                          Gauss-Kronrod rule takes only the embedded one)   */
} gmq_options;

/* gmq_options.flags: record the final partition of the run (every region
 * retired in any sweep, then the regions of the last evaluated sweep), for
 * gmq_partition_copy / gmq_rule_grad.  The list holds up to max_regions
 * regions and adds two region lists to the pool; if it fills up, the run
 * stops with GMQ_CAP_REACHED and no partition is kept. */
#define GMQ_KEEP_PARTITION 1

typedef struct gmq_result {
  double integral;           /* I: retired sums + active regions' I7_r     */
  double error;              /* eps: the same for the regions' eps_r       */
  int64_t regions_evaluated; /* rule applications over all sweeps          */
  int64_t function_evals;    /* regions_evaluated * (2^d + 2d^2 + 2d + 1)  */
  int64_t final_active;      /* regions in the last evaluated sweep        */
  int32_t iterations;        /* sweeps evaluated                           */
  int32_t status;            /* gmq_status of the run                      */
} gmq_result;

/* One record per sweep of the last gmq_integrate call. */
typedef struct gmq_sweep {
  int64_t n;        /* regions evaluated in the sweep                      */
  int64_t n_split;  /* regions bisected (-1 if the loop stopped first)     */
  double I, E;      /* global estimates after the sweep's evaluation       */
  double I_ret, E_ret; /* retired sums after the sweep's classification   */
  double budget;    /* max(abs_tol, rel_tol |I|)                            */
} gmq_sweep;

typedef struct gmq_context gmq_context;

/* Create a context on CUDA device `device`.  pool_bytes_hint > 0 reserves
 * that much device memory up front for the region pool (otherwise the pool
 * grows on demand).  *out receives the context; destroy it with
 * gmq_destroy. */
gmq_status gmq_create(gmq_context **out, int device, size_t pool_bytes_hint);

/* Free the context and the device memory it owns (not a caller pool). */
gmq_status gmq_destroy(gmq_context *ctx);

/* Run all later work of the context on this cudaStream_t (NULL = the legacy
 * default stream).  The stream must belong to the context's device. */
gmq_status gmq_set_stream(gmq_context *ctx, void *cuda_stream);

/* Use caller-owned device memory [dev_ptr, dev_ptr + bytes) as the region
 * pool instead of allocating.  The memory must stay valid until the context
 * is destroyed or another pool is set; dev_ptr must be 256-byte aligned.
 * gmq_integrate then returns GMQ_ERR_OOM if the pool is too small
 * (see gmq_pool_bytes).  Passing NULL returns to library-owned memory. */
gmq_status gmq_set_pool(gmq_context *ctx, void *dev_ptr, size_t bytes);

/* How the FP64 Genz-Malik kernels (gmq_integrate and gmq_eval_rule with
 * GMQ_FP64) evaluate the integrand at a region's nodes (paper Sec. 2: the
 * rule applies f at every node).  Every built-in family is f = g(S), S a
 * chain of per-axis terms phi_j(x_j) combined by + (by * for the product
 * peak), and a node takes each coordinate from one of seven values per axis:
 *   GMQ_EVAL_SEPARABLE (default): phi at the 7d coordinate values once per
 *     region; each node's S from one or two combines of per-axis terms and
 *     partial chains; g at every node;
 *   GMQ_EVAL_NODEWISE: f from each node's coordinates (d operations for S,
 *     then g), as an integrand without that form would be evaluated.
 * Both give every lane mapping the same bits; they differ from each other
 * only in the rounding order of S.  gmq_rule_grad follows it too: the
 * separable mode forms the gradient from per-axis, per-coordinate sums of
 * w g'(S) over the nodes, the node-wise mode differentiates f at every
 * node.  The mixed precision, the Gauss-Kronrod rule and the batched form
 * do not depend on it. */
typedef enum gmq_eval_mode {
  GMQ_EVAL_SEPARABLE = 0,
  GMQ_EVAL_NODEWISE = 1
} gmq_eval_mode;

/* Set the context's gmq_eval_mode (GMQ_ERR_INVALID for another value). */
gmq_status gmq_set_eval_mode(gmq_context *ctx, int32_t mode);

/* Device bytes the region pool needs for dimension dim, max_regions and
 * gmq_options.flags (GMQ_KEEP_PARTITION adds the final-partition list). */
gmq_status gmq_pool_bytes(int32_t dim, int64_t max_regions, int32_t flags,
                          size_t *bytes);

/* Fill opt with defaults: rel_tol 1e-6, abs_tol 1e-16, max_regions 2^22,
 * automatic partition, 1000 sweeps, FP64, volume-share classifier, lanes 0. */
gmq_status gmq_default_options(gmq_options *opt);

/* Integrate (paper Sec. 3 loop).  Synchronous on the context stream.  A
 * positive status still fills *out with the best estimate. */
gmq_status gmq_integrate(gmq_context *ctx, const gmq_problem *prob,
                         const gmq_options *opt, gmq_result *out);

/* Copy up to max records of the last gmq_integrate call's per-sweep trace;
 * *count receives the number of records available. */
gmq_status gmq_last_trace(gmq_context *ctx, gmq_sweep *out, int32_t max,
                          int32_t *count);

/* Final partition of the last gmq_integrate call made with
 * GMQ_KEEP_PARTITION: *count receives its number of regions (-1 if none was
 * kept); up to max regions are copied into the caller's device arrays
 * (layout as for gmq_eval_rule, leading dimension ld >= min(count, max)).
 * The regions tile Omega; their order is the order they left the loop.
 * The list lives in the context's pool until the next gmq_integrate. */
gmq_status gmq_partition_copy(gmq_context *ctx, double *d_center,
                              double *d_halfw, int64_t ld, int64_t max,
                              int64_t *count);

/* ---- batched form ------------------------------------------------------ */

/* gmq_options.flags for gmq_integrate_batch: drive the sweeps from the host
 * (one launch sequence per sweep, status read every few sweeps) instead of
 * one CUDA-graph launch whose while-node runs every sweep on the device. */
#define GMQ_BATCH_HOST_LOOP 2

/* How the last gmq_integrate_batch call ran. */
typedef struct gmq_batch_info {
  int32_t rule_block;   /* threads per block of the rule kernel             */
  int32_t rule_grid;    /* blocks of its persistent grid                    */
  int32_t sweeps;       /* sweeps of the device loop                        */
  int32_t used_graph;   /* 1: ran as one CUDA graph with a while node       */
  int32_t autotuned;    /* 1: this call timed the candidate mappings        */
  int32_t pauses;       /* problem-sweeps deferred because the pool was full */
  int32_t evictions;    /* problems evicted and restarted to make room      */
  int32_t forced_lanes; /* opt->lanes when nonzero, else 0                  */
  int64_t lanes_t1;     /* lists of >= lanes_t1 regions: 1 lane per region  */
  int64_t lanes_t4;     /* >= lanes_t4: 4 lanes                             */
  int64_t lanes_t32;    /* >= lanes_t32: 32 (a warp); shorter lists: 128 (a
                           128-thread block per region)                     */
  int32_t lane_sweeps[4]; /* sweeps run with 1, 4, 32 and 128 lanes        */
  int64_t tune_n[5];    /* list lengths the autotuner timed (0 if unused)   */
  double tune_ms[5][4]; /* rule-kernel time per length and mapping 1/4/32/128 */
  int64_t rule_regions;    /* regions the rule kernels evaluated, including
                              work that evictions later dropped             */
  int64_t carried_regions; /* regions of paused problems carried over
                              unchanged (copied, not evaluated)             */
  int64_t list_regions;    /* sum over sweeps of the list length (the work
                              of the per-sweep sums, classify and split)    */
} gmq_batch_info;

/* Many independent integrals in one device-resident loop (no counterpart in
 * the paper, which integrates one problem at a time).  Every problem runs
 * the paper's loop (Sec. 3) with the same decisions, sums and child order
 * as gmq_integrate gives it alone (with any lanes setting); all of them
 * advance one sweep per iteration, their active regions sharing one region
 * pool of pool_regions regions (0: max(opt->max_regions, 4 x the initial
 * partitions)); opt->max_regions is each problem's own cap.  probs[i] and
 * rel_tols[i] (rel_tols may be NULL: opt->rel_tol for all) describe
 * problem i; results[i] receives its result and status.  When the next
 * sweep of all running problems does not fit in the pool, the problems
 * whose region lists grow are served in index order while they fit; the
 * others are paused for a sweep (their regions are carried over unchanged
 * with their rule outputs and take the same decisions again, which leaves
 * their results unchanged); if nothing can split, the paused problem of
 * highest index is evicted and later restarts from its initial partition
 * (same result again), and a problem that cannot grow even alone stops with
 * GMQ_CAP_REACHED.  The device loop is bounded by 4 x max_iters sweeps
 * (max_iters above 2^28 is rejected with GMQ_ERR_INVALID).
 * Device memory: about pool_regions x (32 dmax + 60) bytes, dmax the
 * largest dimension.
 * opt->precision GMQ_FP64: lanes per region opt->lanes (1, 4, 32 or 128)
 * for every sweep, or with 0 chosen per sweep from the list length by
 * thresholds an autotuner sets on the first call for each largest dimension
 * (it times the four mappings on copies of the initial list at up to five
 * lengths; cached in the context); the results do not depend on the
 * mapping.  opt->precision GMQ_MIXED: one lane per region (opt->lanes must
 * be 0 or 1), one rule launch per family present per sweep, and every
 * problem gets the bits gmq_integrate's mixed form gives it with lanes = 1.
 * Returns GMQ_OK when the batch ran (see the per-problem statuses), or an
 * error. */
gmq_status gmq_integrate_batch(gmq_context *ctx, int32_t count,
                               const gmq_problem *probs, const double *rel_tols,
                               const gmq_options *opt, int64_t pool_regions,
                               gmq_result *results);

/* Launch shape, sweep count and autotuning record of the last batch. */
gmq_status gmq_last_batch_info(gmq_context *ctx, gmq_batch_info *info);

/* Adjoint over a frozen partition (no counterpart in the paper; the
 * differentiation extension).  For the n regions given (typically the
 * final partition of an integration), Q = sum_r vol_r sum_i w_i f(x_i) with
 * the degree-7 Genz-Malik weights, and its exact gradient with respect to
 * the family parameters, dQ/dtheta = sum_r vol_r sum_i w_i df/dtheta(x_i).
 * *integral receives Q; grad (host, 2*dim doubles) receives dQ/da_1..a_dim
 * followed by dQ/du_1..u_dim, each summed over the regions with the
 * pairwise tree.  The discontinuous family's u-derivatives are reported as
 * 0 (its thresholds move a jump, which a fixed partition does not see). */
gmq_status gmq_rule_grad(gmq_context *ctx, const gmq_problem *prob, int64_t n,
                         const double *d_center, const double *d_halfw,
                         int64_t ld, double *integral, double *grad);

/* Seeded Genz parameters (no counterpart in the paper; the paper's
 * integrands use fixed parameters).  SplitMix64 stream with initial state
 * (seed << 16) ^ (family << 8) ^ dim; a_j = top-53-bit doubles in [0,1)
 * rescaled so that sum_j a_j = target_sum, then u_j in [0,1).  a_out and
 * u_out are host arrays of length dim. */
gmq_status gmq_seed_genz(uint64_t seed, int32_t family, int32_t dim,
                         double target_sum, double *a_out, double *u_out);

/* Human-readable name of a status code (static string). */
const char *gmq_status_string(gmq_status s);

/* Name of the CUDA error behind the calling thread's last GMQ_ERR_CUDA or
 * GMQ_ERR_OOM (static string, e.g. "cudaErrorInvalidValue"). */
const char *gmq_last_cuda_error(void);

/* Number of kernels the context has launched since creation. */
gmq_status gmq_launch_count(gmq_context *ctx, int64_t *count);

/* Kernel timing.  While enabled, the context brackets each kernel it
 * launches with CUDA events on its stream and, when the call waits for the
 * stream, adds the measured durations to per-kernel totals.  kernel: 0 rule
 * evaluation (the Genz-Malik, Gauss-Kronrod and gmq_rule_grad kernels), 1
 * global sums (also gmq_rule_grad's row sums), 2 classify, 3 split, 4
 * partition.  `regions` counts the regions the launches processed.  Enabling adds two event
 * records per launch. */
typedef struct gmq_kernel_stats {
  int64_t launches;
  int64_t regions;
  double ms;
} gmq_kernel_stats;

gmq_status gmq_profile_enable(gmq_context *ctx, int32_t on);
gmq_status gmq_profile_reset(gmq_context *ctx);
gmq_status gmq_profile_read(gmq_context *ctx, int32_t kernel, gmq_kernel_stats *out);

/* Measurement aid (no counterpart in the paper): the floating-point issue
 * rate of the context's GPU, measured, as the peak the rule kernels'
 * rooflines are reported against.  precision GMQ_FP64 times FP64
 * operations, GMQ_MIXED FP32 ones; op 0 times fused multiply-adds, 1 adds,
 * 2 multiplies.  One launch of 8 x (SM count) blocks of 256 threads (64
 * warps per SM), each thread running `iters` iterations of 16 independent
 * chains of the operation (1 <= iters <= 2^32), timed with CUDA events on
 * the context stream; the call waits for it.  *lane_ops_per_s receives the
 * lane operations per second (one operation of one thread = one lane
 * operation; a fused multiply-add counts 2 flops), *ms the launch's
 * duration.  Its 8 x (SM count) x 256 x 8-byte result sink is context
 * memory (shared with gmq_rule_grad's working memory). */
gmq_status gmq_probe_fp_rate(gmq_context *ctx, int32_t precision, int32_t op, int64_t iters,
                             double *lane_ops_per_s, double *ms);

/* ---- step-level calls on caller device memory (one sweep's pieces) ---- */

/* Rule evaluation (paper Sec. 2) on n regions.  Outputs, each of length n:
 * d_integral[r] = I7_r; d_error[r] = eps_r, the estimator's value
 * (gmq_estimator: |I7_r - I5_r| or the null-rule estimate); d_volfrac[r] =
 * vol_r / vol(Omega) with vol_r = prod_k 2 h_k and vol(Omega) from the
 * problem's lo, hi; d_axis[r] = split axis in bits 0..6, bit 7 set when
 * bisecting along that axis cannot move the centre (round-off guard).
 * precision: gmq_precision; lanes: 0, 1, 4, 32 or (FP64) 128 as in
 * gmq_options; estimator: gmq_estimator.
 * d_volfrac may be NULL. */
gmq_status gmq_eval_rule(gmq_context *ctx, const gmq_problem *prob,
                         int32_t precision, int32_t lanes, int32_t estimator, int64_t n,
                         const double *d_center, const double *d_halfw,
                         int64_t ld, double *d_integral, double *d_error,
                         double *d_volfrac, uint8_t *d_axis);

/* The tensor-product Gauss-Kronrod rule (gmq_rule) on n regions, FP64, one
 * warp per region; outputs as for gmq_eval_rule with d_integral[r] = I_K
 * (the 15^dim-node value) and d_error[r] = |I_K - I_G|.  dim <=
 * GMQ_GK_MAX_DIM, else GMQ_ERR_INVALID.  Synchronous on the context stream. */
gmq_status gmq_eval_rule_gk(gmq_context *ctx, const gmq_problem *prob, int64_t n,
                            const double *d_center, const double *d_halfw,
                            int64_t ld, double *d_integral, double *d_error,
                            double *d_volfrac, uint8_t *d_axis);

/* The library's 1-D Gauss-Kronrod tables on [-1, 1] (host memory, 45
 * doubles): out[0..15) the 15 nodes in ascending order, out[15..30) their
 * Kronrod weights, out[30..45) the Gauss weights (0 at the 8 Kronrod-only
 * nodes).  Computed on the host (Newton iteration for the Legendre zeros,
 * bisection for the zeros of the Stieltjes polynomial, an 8 x 8 solve for
 * the Kronrod weights); no device work. */
gmq_status gmq_gk_table(double *out);

/* The library's null-rule table for dimension dim (host memory, 20
 * doubles; GMQ_EST_NULL_RULES): out[5k + c] is null rule N_{k+1}'s weight
 * per node of class c (centre, +-lambda2 e_k, +-lambda3 e_k, pairs,
 * corners), unit volume; rows of degree 5, 3, 3, 1 (for dim 1 the third
 * row is zero).  Computed on the host; no device work. */
gmq_status gmq_null_rule_table(int32_t dim, double *out);

/* The FP64 exponential the built-in integrands use (Tang's table-driven
 * method; within about one ulp), on n device values: d_y[i] = exp(d_x[i]).
 * No counterpart in the paper; exposed so that its accuracy can be tested
 * against the CUDA and host libraries.  Synchronous on the context
 * stream. */
gmq_status gmq_math_exp(gmq_context *ctx, int64_t n, const double *d_x,
                        double *d_y);

/* The FP64 reciprocal the product-peak and corner-peak integrands use (the
 * hardware approximation refined by two Newton-Raphson steps; within one
 * ulp), on n device values: d_y[i] = 1 / d_x[i].  Exposed for testing, as
 * gmq_math_exp. */
gmq_status gmq_math_rcp(gmq_context *ctx, int64_t n, const double *d_x,
                        double *d_y);

/* The FP64 cosine the oscillatory integrand uses (table-driven; absolute
 * error within a few units of 2^-53), on n device values: d_y[i] =
 * cos(d_x[i]).  Exposed for testing, as gmq_math_exp. */
gmq_status gmq_math_cos(gmq_context *ctx, int64_t n, const double *d_x,
                        double *d_y);

/* Classification and bisection of one sweep (paper Sec. 3) given the rule
 * outputs above and the sweep's budget = max(abs_tol, rel_tol |I|).
 * Region r is retired if eps_r <= budget * volfrac_r (GMQ_VOLUME_SHARE) or
 * eps_r <= rel_tol |I_r| (GMQ_LOCAL_REL), or eps_r <= 50 * 2^-53 |I_r|, or
 * bit 7 of d_axis[r] is set; otherwise it is split.  The left children of
 * the split regions, in input order, are written to slots [0, n_split) of
 * the output arrays and the right children to [n_split, 2 n_split).
 * If 2 n_split > cap_out nothing is written and GMQ_CAP_REACHED is returned
 * (n_split and the sums are still reported).  d_flags (may be NULL)
 * receives 1 for split, 0 for retired.  *retired_integral and
 * *retired_error receive the pairwise-tree sums over the list of the
 * retired regions' I_r and eps_r (split regions count as zero). */
gmq_status gmq_classify_split(gmq_context *ctx, int32_t dim, int64_t n,
                              const double *d_center, const double *d_halfw,
                              int64_t ld, const double *d_integral,
                              const double *d_error, const double *d_volfrac,
                              const uint8_t *d_axis, double budget,
                              double rel_tol, int32_t classifier,
                              double *d_center_out, double *d_halfw_out,
                              int64_t ld_out, int64_t cap_out,
                              uint8_t *d_flags, int64_t *n_split,
                              double *retired_integral, double *retired_error);

/* Pairwise-tree sum of d_v[0..n): sum(range) = sum(left half) +
 * sum(right half) over the range zero-padded to a power of two.  The same
 * order is used for every global sum of the loop. */
gmq_status gmq_tree_sum(gmq_context *ctx, int64_t n, const double *d_v,
                        double *sum);

/* Initial uniform partition (paper Sec. 3): s^dim boxes of equal size,
 * the axis-0 index fastest; along axis k box i has h_k = (hi_k - lo_k)/(2s)
 * and c_k = lo_k + (2i + 1) h_k.  ld >= s^dim. */
gmq_status gmq_partition(gmq_context *ctx, int32_t dim, const double *lo,
                         const double *hi, int32_t s, double *d_center,
                         double *d_halfw, int64_t ld);

/* ---- allocation-free variant ------------------------------------------ */

/* Longest input of gmq_tree_sum_noalloc: 2^23 values (8192 tiles). */
#define GMQ_NOALLOC_MAX_N ((int64_t)1 << 23)

/* The pairwise-tree sum of gmq_tree_sum (same order, same result) without
 * any device allocation.  The paper has no counterpart: this call exists for
 * callers that cannot allocate device memory at the point where they need
 * the sum -- code whose device memory is wholly owned by its own allocator
 * or a fixed budget reserved at start-up, and code that cannot afford the
 * device-wide synchronisation that cudaMalloc and cudaFree may cause in the
 * middle of its work.  It needs no gmq_context (creating one allocates).
 *
 * Arguments: device is the CUDA device of d_v, d_sum and the stream; d_v
 * holds n doubles (device memory, read only); d_sum receives the sum (one
 * double of device memory); cuda_stream is the cudaStream_t to run on (NULL
 * = the legacy default stream).  The call only enqueues work on that
 * stream: the sum is in *d_sum once the stream reaches that point.
 *
 * Working memory: a file-scope static device array of about 64 KiB (the
 * last-block ticket and one partial sum per 1024-value tile), which every
 * device that loads the library keeps until the process exits.  Every call
 * looks up the array's device address on `device` (cudaGetSymbolAddress,
 * which allocates nothing); the first lookup on a device may load the
 * library's device code there, so make the first call on a device before
 * any stream capture.  All calls share the one array, and each call clears
 * the ticket it needs on its own stream, so calls whose work overlaps on the
 * GPU (different streams, or several host threads) race and must be
 * serialised by the caller.
 *
 * Errors: GMQ_ERR_TOO_LARGE if n > GMQ_NOALLOC_MAX_N (nothing is enqueued);
 * GMQ_ERR_INVALID for a negative n, a NULL pointer, a bad device, or d_v /
 * d_sum not in that device's memory; GMQ_ERR_CUDA if the address lookup,
 * the memset or the launch fails (the CUDA error is cleared before the
 * call returns).  The
 * call makes no cudaMalloc, cudaFree or other allocating call. */
gmq_status gmq_tree_sum_noalloc(int32_t device, int64_t n, const double *d_v,
                                double *d_sum, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GMQ_H */
