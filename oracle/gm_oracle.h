/*
 * gm_oracle.h -- plain FP64 CPU oracle of the adaptive Genz-Malik quadrature.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: every constant below is
 * recomputed here from the published formulas.
 *
 * Region layout in this oracle is plain array-of-structures: region r has
 * centre c[r*d + k] and half-width h[r*d + k], k = 0..d-1.
 */
#ifndef GM_ORACLE_H
#define GM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* f(x) for x in R^d; ctx is opaque user data. */
typedef double (*or_integrand)(const double *x, int d, const void *ctx);

/* Built-in integrand families (paper Sec. 4 test functions and the Genz
 * families they instantiate). */
enum {
  OR_OSCILLATORY = 0,   /* cos(2*pi*u_1 + sum a_j x_j)                    */
  OR_PRODUCT_PEAK = 1,  /* prod 1/(a_j^-2 + (x_j-u_j)^2)                  */
  OR_CORNER_PEAK = 2,   /* (1 + sum a_j x_j)^-(d+1)                       */
  OR_GAUSSIAN = 3,      /* exp(-sum a_j^2 (x_j-u_j)^2)                    */
  OR_C0 = 4,            /* exp(-sum a_j |x_j-u_j|)                        */
  OR_DISCONTINUOUS = 5, /* 0 if any x_j > u_j, else exp(sum a_j x_j)      */
  OR_POLY_SUMSQ11 = 6   /* (sum x_j^2)^11                                 */
};

typedef struct {
  int32_t family;
  int32_t d;
  const double *a; /* length d */
  const double *u; /* length d */
} or_family;

/* Result of the rule on one region. */
typedef struct {
  double i7, i5, err; /* degree-7 value, embedded degree-5 value, |i7-i5|  */
  double s[5];        /* class sums S1..S5                                  */
  double sabs[5];     /* sums of |f| per class (magnitude of the terms)     */
  double vol;         /* prod_k 2 h_k                                       */
  double f0;          /* f at the centre                                    */
  int32_t axis;       /* chosen split axis                                  */
  int32_t axis_tie;   /* 1 if the axis choice is a near-tie                 */
  int32_t flat;       /* 1 if every fourth difference is at noise level     */
  int32_t split_bad;  /* 1 if bisection along axis is not representable     */
} or_rule_out;

typedef struct {
  double rel_tol;
  double abs_tol;
  int64_t max_regions;
  int32_t init_splits; /* 0 = automatic */
  int32_t max_iters;   /* 0 = 1000 */
  int32_t classifier;  /* 0 = volume share, 1 = local relative */
  int32_t rule;        /* 0 = Genz-Malik, 1 = tensor-product Gauss-Kronrod */
  const double *gk;    /* rule 1: the 45-double table of or_rule_gk        */
  int32_t estimator;   /* 0 = |I7 - I5|, 1 = null rules (Genz-Malik only)  */
  const double *null_w; /* estimator 1: the 4 x 5 table of or_null_estimate */
} or_options;

/* Result of the tensor-product Gauss-Kronrod rule on one region. */
typedef struct {
  double ik, ig, err; /* K15^d value, G7^d value, |ik - ig|                 */
  double vol;         /* prod_k 2 h_k                                       */
  double scale;       /* prod_k h_k * sum over nodes of |K weight * f|      */
  int32_t axis, axis_tie, flat, split_bad;
} or_gk_out;

typedef struct {
  double integral, error;
  int64_t regions_evaluated, function_evals, final_active;
  int32_t iterations, status;
  int64_t near_ties; /* decisions within the near-tie band over the run */
} or_result;

/* Per-sweep trace record (optional). */
typedef struct {
  int64_t n, n_split, near_ties;
  double I, E, I_ret, E_ret, budget;
} or_trace;

/* Rule description. */
int64_t or_num_nodes(int d);
void or_lambdas(double lam[4]);                 /* lambda2..lambda5          */
void or_weights(int d, double w7[5], double w5[5]);

/* One built-in integrand at one point; ctx is an or_family*. */
double or_family_eval(const double *x, int d, const void *ctx);

/* Genz-Malik degree-7 rule with embedded degree-5 rule on one region.
 * D (length d, may be NULL) receives the fourth differences. */
void or_rule(int d, const double *c, const double *h, or_integrand f,
             const void *ctx, double *D, or_rule_out *out);

/* The rule over n regions of a built-in family (AoS c, h).  Output arrays
 * of length n; any may be NULL. */
void or_rule_regions(const or_family *fam, int64_t n, const double *c,
                     const double *h, double *i7, double *i5, double *err,
                     double *vol, int32_t *axis, int32_t *axis_tie,
                     int32_t *split_bad, double *i7abs);

/* Null-rule error estimate (Berntsen, Espelid & Genz 1991, the heuristic
 * the paper's Sec. 2 cites; its form here is a reading, see gm_oracle.c).
 * null_w: 4 x 5 per-node weights of the null rules N1..N4 per node class
 * (unit volume, row-major; oracle/null_rules.py); rule: the region's rule
 * output (class sums, class magnitude sums, volume). */
typedef struct {
  double nul[4];    /* N_k = vol * sum_c null_w[k][c] S_c                     */
  double e[3];      /* |N1|, sqrt(N2^2 + N3^2), |N4|                          */
  double r;         /* max(e1 / e2, e2 / e3): decay per degree step          */
  double est;       /* the error estimate                                     */
  double est_alt;   /* the estimate on the other side of the r = 1 boundary  */
  double noise;     /* rounding band of the null values: 1e-13 vol sum_c max_k |null_w[k][c]| A_c */
  double band;      /* resulting rounding band of est (interval bound)       */
  int32_t regime;   /* 0: r >= 1 (not asymptotic), 1: r < 1 (asymptotic)     */
  int32_t regime_tie; /* the e_k's rounding band reaches across r = 1        */
} or_null_out;

void or_null_estimate(const or_rule_out *rule, const double *null_w, or_null_out *out);

/* The rule over n regions with the chosen estimator (null_w == NULL: the
 * embedded |I7 - I5|, else the null-rule estimate), as the loop uses it.
 * err_band (may be NULL) receives each error value's rounding band: the
 * half-width within which two correct FP64 implementations may differ. */
void or_rule_regions_est(const or_family *fam, int64_t n, const double *c,
                         const double *h, const double *null_w, double *i7,
                         double *err, double *vol, int32_t *axis,
                         int32_t *axis_tie, int32_t *split_bad, double *scale,
                         double *err_band, double *err_alt);

/* Pairwise (binary tree over a zero-padded power of two) sum. */
/* Tensor-product Gauss-Kronrod (7, 15) rule on one region (the paper's
 * Sec. 3 names the rule, not its order or its split axis; these are
 * readings).  gk: 15 nodes of [-1, 1] in ascending order, then their K15
 * weights, then the G7 weights (0 at the 8 Kronrod-only nodes).  Nodes
 * x = fma(node, h_k, c_k) over all 15^d index tuples, axis 0 fastest;
 * ik = prod h_k sum w_K f, ig the same with the G7 weights, err = |ik - ig|.
 * E_k (written to E if not NULL) = prod h_k |sum (prod_{j != k} w_K)(w_K,k -
 * w_G,k) f|: the error estimate in direction k (G7 along axis k, K15 along
 * the others, against K15 everywhere); the split axis is argmax E_k, the
 * lowest index on ties, or the widest axis when every E_k is below 1e-11
 * of scale (rounding noise).  d <= 6. */
int64_t or_gk_nodes(int d);
void or_rule_gk(int d, const double *c, const double *h, or_integrand f,
                const void *ctx, const double *gk, double *E, or_gk_out *out);
void or_rule_gk_regions(const or_family *fam, int64_t n, const double *c,
                        const double *h, const double *gk, double *ik,
                        double *ig, double *err, double *vol, int32_t *axis,
                        int32_t *axis_tie, int32_t *split_bad, double *scale);

double or_pairwise_sum(const double *v, int64_t n);

/* Initial uniform partition: returns s used; writes s^d regions. */
int32_t or_auto_splits(int d, int64_t cap);
int64_t or_partition(int d, const double *lo, const double *hi, int32_t s,
                     double *c, double *h);

/* Classification of one sweep.  flags[r] = 1 split, 0 retire.  Returns the
 * number of split regions; retired sums and near-tie count via pointers.
 * scale (may be NULL) is the per-region magnitude used for the near-tie
 * band; err_band (may be NULL) replaces its 1e-13 scale term by the given
 * per-region band of err. */
int64_t or_classify(int d, int64_t n, const double *i7, const double *err,
                    const double *vol, const int32_t *split_bad,
                    const double *scale, double vol_omega, double budget,
                    double rel_tol, int32_t classifier, uint8_t *flags,
                    double *ret_i, double *ret_e, int64_t *near_ties);
int64_t or_classify_band(int d, int64_t n, const double *i7, const double *err,
                         const double *vol, const int32_t *split_bad,
                         const double *scale, const double *err_band,
                         double vol_omega, double budget, double rel_tol,
                         int32_t classifier, uint8_t *flags, double *ret_i,
                         double *ret_e, int64_t *near_ties);

/* Bisection + compaction: left children of split regions in input order at
 * [0, n_split), right children at [n_split, 2 n_split). */
int64_t or_bisect(int d, int64_t n, const double *c, const double *h,
                  const int32_t *axis, const uint8_t *flags, double *c_out,
                  double *h_out);

/* Derivative of a built-in integrand with respect to parameter k
 * (k < d: a_k, k >= d: u_{k-d}); ctx is an or_deriv_ctx*. */
typedef struct {
  const or_family *fam;
  int32_t k;
} or_deriv_ctx;
double or_family_deriv(const double *x, int d, const void *ctx);

/* Frozen-partition quadrature Q = sum_r I7_r and its gradient: the same rule
 * applied to each derivative integrand, summed over the regions with the
 * pairwise tree.  grad has 2d entries (a_1..a_d, u_1..u_d). */
void or_rule_grad(const or_family *fam, int64_t n, const double *c,
                  const double *h, double *grad, double *integral);

/* Like or_integrate, and also returns the final partition (every retired region followed by the regions of
 * the last evaluated sweep) in c_out/h_out (capacity max_leaves regions);
 * *n_leaves receives its size, or -1 if it did not fit. */
int32_t or_integrate_partition(const or_family *fam, const double *lo,
                               const double *hi, const or_options *opt,
                               or_result *res, double *c_out, double *h_out,
                               int64_t max_leaves, int64_t *n_leaves);

/* The whole adaptive loop.  trace (may be NULL) receives up to max_trace
 * records.  Status codes: 0 converged, 1 region cap reached, 2 iteration
 * limit, 3 every region retired before the tolerance was met,
 * -1 invalid argument, -2 out of memory, -4 non-finite integrand. */
int32_t or_integrate(const or_family *fam, const double *lo, const double *hi,
                     const or_options *opt, or_result *res, or_trace *trace,
                     int32_t max_trace);

#ifdef __cplusplus
}
#endif
#endif
