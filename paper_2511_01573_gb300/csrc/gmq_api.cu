// gmq_api.cu -- host side of the library: the C ABI declared in gmq.h, the
// context and its region pool, and the adaptive loop that drives the sweep
// kernels (paper Sec. 3, Fig. 1a; stopping rule paper Sec. 4).
//
// Per sweep the host enqueues, on the context stream:
//   rule evaluation (K1) -> global sums + convergence test -> classify ->
//   split into the other half of the ping-pong pool,
// then copies the 80-byte device status to pinned host memory and waits on
// it: the only host<->device traffic of a sweep.  Every kernel after the
// sums checks the device status and returns at once when the loop is done,
// so a converged sweep does no classification or splitting work.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gm_adjoint.cuh"
#include "gm_gk.cuh"
#include "gm_rule.cuh"
#include "gmq_common.cuh"
#include "gm_batch.cuh"
#include "sweep_kernels.cuh"

using namespace gmq;

namespace gmq {
template <int FAM>
cudaError_t launch_rule_family(int precision, int T, const RuleArgs& A, cudaStream_t s);
extern template cudaError_t launch_rule_grad_family<GMQ_OSCILLATORY>(const GradArgs&, cudaStream_t);
extern template cudaError_t launch_rule_grad_family<GMQ_PRODUCT_PEAK>(const GradArgs&, cudaStream_t);
extern template cudaError_t launch_rule_grad_family<GMQ_CORNER_PEAK>(const GradArgs&, cudaStream_t);
extern template cudaError_t launch_rule_grad_family<GMQ_GAUSSIAN>(const GradArgs&, cudaStream_t);
extern template cudaError_t launch_rule_grad_family<GMQ_C0>(const GradArgs&, cudaStream_t);
extern template cudaError_t launch_rule_grad_family<GMQ_DISCONTINUOUS>(const GradArgs&, cudaStream_t);
extern template cudaError_t launch_rule_grad_family<GMQ_POLY_SUMSQ11>(const GradArgs&, cudaStream_t);
extern template cudaError_t launch_rule_gk_family<GMQ_OSCILLATORY>(const GkArgs&, cudaStream_t);
extern template cudaError_t launch_rule_gk_family<GMQ_PRODUCT_PEAK>(const GkArgs&, cudaStream_t);
extern template cudaError_t launch_rule_gk_family<GMQ_CORNER_PEAK>(const GkArgs&, cudaStream_t);
extern template cudaError_t launch_rule_gk_family<GMQ_GAUSSIAN>(const GkArgs&, cudaStream_t);
extern template cudaError_t launch_rule_gk_family<GMQ_C0>(const GkArgs&, cudaStream_t);
extern template cudaError_t launch_rule_gk_family<GMQ_DISCONTINUOUS>(const GkArgs&, cudaStream_t);
extern template cudaError_t launch_rule_gk_family<GMQ_POLY_SUMSQ11>(const GkArgs&, cudaStream_t);
}

struct gmq_context {
  int device = 0;
  int sm_count = 1;
  cudaStream_t stream = nullptr;
  char* own = nullptr;
  size_t own_bytes = 0;
  char* ext = nullptr;
  size_t ext_bytes = 0;
  char* scratch = nullptr;
  size_t scratch_bytes = 0;
  DevStatus* h_status = nullptr;  // pinned, large enough for a BatchState too
  std::vector<gmq_sweep> trace;
  int64_t launches = 0;
  // final partition of the last integration (GMQ_KEEP_PARTITION)
  int64_t part_count = -1;
  int part_d = 0;
  int64_t part_ld = 0;
  const double* part_c = nullptr;
  const double* part_h = nullptr;
  // working memory of gmq_rule_grad
  char* gscratch = nullptr;
  GkConst* gk_dev = nullptr;  // device copy of the Gauss-Kronrod tables
  size_t gscratch_bytes = 0;
  // batched form: autotuned lanes-per-region thresholds per largest dimension
  int tuned[GMQ_MAX_DIM + 1] = {};
  long long tuned_t1[GMQ_MAX_DIM + 1] = {};
  long long tuned_t4[GMQ_MAX_DIM + 1] = {};
  long long tuned_t32[GMQ_MAX_DIM + 1] = {};
  gmq_batch_info last_batch = {};
  int eval_mode = GMQ_EVAL_SEPARABLE;     // gmq_set_eval_mode
  cudaStream_t capture_stream = nullptr;  // private stream for graph capture
  // kernel timing (gmq_profile_*)
  bool prof_on = false;
  bool ev_made = false;
  cudaEvent_t ev[5][2] = {};
  bool pending[5] = {};
  int64_t pend_regions[5] = {};
  gmq_kernel_stats stats[5] = {};
};

namespace {

constexpr int64_t kMaxRegions = (int64_t)1 << 30;

// Round-off guard (paper Sec. 3): a region whose error estimate is below
// g u |I7_r| is at the rounding level of its own rule value and is retired.
// FP64: g = 50, u = 2^-53.  Mixed form (FP32 node values): g = 4, u = 2^-24,
// about twice the spread that FP32 node values leave in |I7 - I5|.
constexpr double kGuardFp64 = 50.0 * 0x1p-53;
constexpr double kGuardMixed = 4.0 * 0x1p-24;

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// NVTX range for timeline tools (a no-op unless a tool is attached): one per
// public call and one per sweep of the single-integral loop.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
  ~NvtxRange() { nvtxRangePop(); }
};

int64_t num_nodes(int d) { return ((int64_t)1 << d) + 2 * (int64_t)d * d + 2 * (int64_t)d + 1; }

// Region pool of one integration: two region lists (ping-pong), the rule
// outputs, the decision bytes, per-tile arrays, the device status and, with
// GMQ_KEEP_PARTITION, the final-partition list.
struct PoolLayout {
  int64_t ld = 0, nb = 0;
  size_t cA = 0, hA = 0, cB = 0, hB = 0, i7 = 0, err = 0, vf = 0, axis = 0, flags = 0;
  size_t cnt = 0, off = 0, ba = 0, bb = 0, st = 0, cL = 0, hL = 0, total = 0;
};

PoolLayout pool_layout(int d, int64_t cap, int flags) {
  PoolLayout L;
  L.ld = (cap + 31) / 32 * 32;
  L.nb = (cap + kTile - 1) / kTile;
  size_t p = 0;
  const size_t list = align256(sizeof(double) * (size_t)d * (size_t)L.ld);
  const size_t vec = align256(sizeof(double) * (size_t)L.ld);
  const size_t bytes = align256((size_t)L.ld);
  L.cA = p; p += list;
  L.hA = p; p += list;
  L.cB = p; p += list;
  L.hB = p; p += list;
  L.i7 = p; p += vec;
  L.err = p; p += vec;
  L.vf = p; p += vec;
  L.axis = p; p += bytes;
  L.flags = p; p += bytes;
  L.cnt = p; p += align256(sizeof(int) * (size_t)L.nb);
  L.off = p; p += align256(sizeof(long long) * (size_t)L.nb);
  L.ba = p; p += align256(sizeof(double) * (size_t)L.nb);
  L.bb = p; p += align256(sizeof(double) * (size_t)L.nb);
  L.st = p; p += align256(sizeof(DevStatus));
  if (flags & GMQ_KEEP_PARTITION) {
    L.cL = p; p += list;
    L.hL = p; p += list;
  }
  L.total = p;
  return L;
}

// Null rules for the null-rule error estimate (Berntsen, Espelid & Genz
// 1991, cited by the paper's Sec. 2): four fully symmetric null rules on the
// rule's five node classes, of degrees 5, 3, 3 and 1, mutually orthogonal
// for <u, v> = sum over nodes u v = sum_c n_c u_c v_c, each with the norm of
// the degree-7 weights.  Built here from the conditions' side: with g_m the
// class sums of monomial m divided by the class sizes (g_1, g_{x1^2},
// g_{x1^4}, g_{x1^2 x2^2}), a rule v annihilates m iff <v, g_m> = 0, so
//   - N4 spans the degree-1 null rules orthogonal to the degree-3 ones:
//     g_{x1^2} made orthogonal to g_1;
//   - N2, N3 span the degree-3 null rules orthogonal to the degree-5 ones:
//     g_{x1^4}, g_{x1^2 x2^2} made orthogonal to g_1, g_{x1^2} and each
//     other (d = 1 has no x2 and no pair class: N3 = 0);
//   - N1 spans the degree-5 null rules: w7 - w5 (the difference of the two
//     embedded rules, both exact to degree 5).
// Gram-Schmidt in that order (modified, twice for stability), then each
// scaled to |w7|.  nw: 4 x 5, row k = N_{k+1}'s weight per node of class c.
void null_rule_weights(int d, const double* w7, const double* w5, double* nw) {
  const double l2 = 9.0 / 70.0, l3 = 9.0 / 10.0, l5 = 9.0 / 19.0;  // lambda^2 (lambda4 = lambda3)
  const double n[5] = {1.0, 2.0 * d, 2.0 * d, 2.0 * d * (d - 1), std::ldexp(1.0, d)};
  auto dot = [&](const double* u, const double* v) {
    double t = 0.0;
    for (int c = 0; c < 5; ++c) t += n[c] * u[c] * v[c];
    return t;
  };
  auto divide = [&](double* g) {
    for (int c = 0; c < 5; ++c) g[c] = n[c] > 0.0 ? g[c] / n[c] : 0.0;
  };
  double g[4][5] = {
      {1.0, 2.0 * d, 2.0 * d, 2.0 * d * (d - 1), n[4]},
      {0.0, 2.0 * l2, 2.0 * l3, 4.0 * (d - 1) * l3, n[4] * l5},
      {0.0, 2.0 * l2 * l2, 2.0 * l3 * l3, 4.0 * (d - 1) * l3 * l3, n[4] * l5 * l5},
      {0.0, 0.0, 0.0, 4.0 * l3 * l3, n[4] * l5 * l5}};
  const int ng = d >= 2 ? 4 : 3;
  for (int m = 0; m < ng; ++m) divide(g[m]);
  for (int m = 0; m < ng; ++m)
    for (int pass = 0; pass < 2; ++pass)
      for (int q = 0; q < m; ++q) {
        const double f = dot(g[m], g[q]) / dot(g[q], g[q]);
        for (int c = 0; c < 5; ++c) g[m][c] -= f * g[q][c];
      }
  const double norm7 = std::sqrt(dot(w7, w7));
  double rows[4][5] = {};
  for (int c = 0; c < 5; ++c) rows[0][c] = w7[c] - w5[c];
  if (d == 1) rows[0][3] = 0.0;
  for (int c = 0; c < 5; ++c) {
    rows[1][c] = g[2][c];
    rows[2][c] = d >= 2 ? g[3][c] : 0.0;
    rows[3][c] = g[1][c];
  }
  for (int k = 0; k < 4; ++k) {
    const double nn = dot(rows[k], rows[k]);
    const double f = nn > 0.0 ? norm7 / std::sqrt(nn) : 0.0;
    for (int c = 0; c < 5; ++c) nw[k * 5 + c] = rows[k][c] * f;
  }
}

RuleConst rule_const(int d, const double* lo, const double* hi, int estimator = GMQ_EST_EMBEDDED) {
  RuleConst R;
  const double dd = (double)d;
  R.lam2 = std::sqrt(9.0 / 70.0);
  R.lam3 = std::sqrt(9.0 / 10.0);
  R.lam5 = std::sqrt(9.0 / 19.0);
  R.w7[0] = (12824.0 - 9120.0 * dd + 400.0 * dd * dd) / 19683.0;
  R.w7[1] = 980.0 / 6561.0;
  R.w7[2] = (1820.0 - 400.0 * dd) / 19683.0;
  R.w7[3] = 200.0 / 19683.0;
  R.w7[4] = 6859.0 / (19683.0 * std::ldexp(1.0, d));
  R.w5[0] = (729.0 - 950.0 * dd + 50.0 * dd * dd) / 729.0;
  R.w5[1] = 245.0 / 486.0;
  R.w5[2] = (265.0 - 100.0 * dd) / 1458.0;
  R.w5[3] = 25.0 / 729.0;
  R.w5[4] = 0.0;
  R.ratio = 1.0 / 7.0;
  double v = 1.0;
  for (int k = 0; k < d; ++k) {
    const double l = lo ? lo[k] : 0.0, h = hi ? hi[k] : 1.0;
    v = v * (h - l);
  }
  R.vol_omega = v;
  R.nodes = num_nodes(d);
  R.estimator = estimator;
  for (int k = 0; k < 20; ++k) R.nw[k] = 0.0;
  if (estimator == GMQ_EST_NULL_RULES) null_rule_weights(d, R.w7, R.w5, R.nw);
  return R;
}

FamParams fam_params(const gmq_problem* p) {
  FamParams P;
  std::memset(&P, 0, sizeof(P));
  P.d = p->dim;
  P.family = p->family;
  for (int j = 0; j < p->dim; ++j) {
    P.a[j] = p->a ? p->a[j] : 0.0;
    P.u[j] = p->u ? p->u[j] : 0.0;
    if (p->family == GMQ_PRODUCT_PEAK) P.b[j] = 1.0 / (P.a[j] * P.a[j]);
    if (p->family == GMQ_GAUSSIAN) P.b[j] = P.a[j] * P.a[j];
  }
  if (p->family == GMQ_OSCILLATORY) P.c0 = 2.0 * M_PI * P.u[0];
  return P;
}

gmq_status validate_problem(const gmq_problem* p) {
  if (!p) return GMQ_ERR_INVALID;
  if (p->dim < 1 || p->dim > GMQ_MAX_DIM) return GMQ_ERR_INVALID;
  if (p->family < 0 || p->family >= GMQ_NUM_FAMILIES) return GMQ_ERR_INVALID;
  if (p->family != GMQ_POLY_SUMSQ11 && (!p->a || !p->u)) return GMQ_ERR_INVALID;
  for (int k = 0; k < p->dim; ++k) {
    const double l = p->lo ? p->lo[k] : 0.0, h = p->hi ? p->hi[k] : 1.0;
    if (!std::isfinite(l) || !std::isfinite(h) || !(h > l)) return GMQ_ERR_INVALID;
    if (p->a && !std::isfinite(p->a[k])) return GMQ_ERR_INVALID;
    if (p->u && !std::isfinite(p->u[k])) return GMQ_ERR_INVALID;
  }
  return GMQ_OK;
}

int auto_splits(int d, int64_t cap) {
  const int64_t lim = std::min<int64_t>(cap, 4096);
  int s = 1;
  for (;;) {
    int64_t p = 1;
    bool over = false;
    for (int k = 0; k < d; ++k) {
      p *= (s + 1);
      if (p > lim) {
        over = true;
        break;
      }
    }
    if (over) break;
    ++s;
  }
  return s;
}

// Threads per region for a sweep of n regions: one thread per region once
// there are enough regions to give every SM about eight warps; otherwise
// split each region's nodes over 4 or 32 lanes.
// Lanes per region for a sweep of n regions: enough threads to fill the
// GPU (about 256 per SM), a thread per region when the list alone does;
// a 128-thread block per region (FP64 only) for very short lists of
// regions with many nodes.
int choose_lanes(int req, int64_t n, int d, int sms, int precision) {
  if (req) return req;
  const int64_t nodes = num_nodes(d);
  const int64_t want = (int64_t)sms * 256;
  if (n >= want || nodes < 16) return 1;
  if (n * 4 >= want || nodes < 128) return 4;
  if (n * 32 >= want || nodes < 1024 || precision != GMQ_FP64) return 32;
  return 128;
}

cudaError_t launch_rule(int fam, int precision, int T, const RuleArgs& A, cudaStream_t s) {
  switch (fam) {
    case GMQ_OSCILLATORY: return launch_rule_family<GMQ_OSCILLATORY>(precision, T, A, s);
    case GMQ_PRODUCT_PEAK: return launch_rule_family<GMQ_PRODUCT_PEAK>(precision, T, A, s);
    case GMQ_CORNER_PEAK: return launch_rule_family<GMQ_CORNER_PEAK>(precision, T, A, s);
    case GMQ_GAUSSIAN: return launch_rule_family<GMQ_GAUSSIAN>(precision, T, A, s);
    case GMQ_C0: return launch_rule_family<GMQ_C0>(precision, T, A, s);
    case GMQ_DISCONTINUOUS: return launch_rule_family<GMQ_DISCONTINUOUS>(precision, T, A, s);
    case GMQ_POLY_SUMSQ11: return launch_rule_family<GMQ_POLY_SUMSQ11>(precision, T, A, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_launch_rule_mixed(int fam, const BatchArgs& B, int grid, cudaStream_t s) {
  switch (fam) {
    case GMQ_OSCILLATORY: return batch_launch_rule_mixed_family<GMQ_OSCILLATORY>(B, grid, s);
    case GMQ_PRODUCT_PEAK: return batch_launch_rule_mixed_family<GMQ_PRODUCT_PEAK>(B, grid, s);
    case GMQ_CORNER_PEAK: return batch_launch_rule_mixed_family<GMQ_CORNER_PEAK>(B, grid, s);
    case GMQ_GAUSSIAN: return batch_launch_rule_mixed_family<GMQ_GAUSSIAN>(B, grid, s);
    case GMQ_C0: return batch_launch_rule_mixed_family<GMQ_C0>(B, grid, s);
    case GMQ_DISCONTINUOUS: return batch_launch_rule_mixed_family<GMQ_DISCONTINUOUS>(B, grid, s);
    case GMQ_POLY_SUMSQ11: return batch_launch_rule_mixed_family<GMQ_POLY_SUMSQ11>(B, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_launch_rule64(int fam, const BatchArgs& B, int grid, cudaStream_t s) {
  switch (fam) {
    case GMQ_OSCILLATORY: return batch_launch_rule64_family<GMQ_OSCILLATORY>(B, grid, s);
    case GMQ_PRODUCT_PEAK: return batch_launch_rule64_family<GMQ_PRODUCT_PEAK>(B, grid, s);
    case GMQ_CORNER_PEAK: return batch_launch_rule64_family<GMQ_CORNER_PEAK>(B, grid, s);
    case GMQ_GAUSSIAN: return batch_launch_rule64_family<GMQ_GAUSSIAN>(B, grid, s);
    case GMQ_C0: return batch_launch_rule64_family<GMQ_C0>(B, grid, s);
    case GMQ_DISCONTINUOUS: return batch_launch_rule64_family<GMQ_DISCONTINUOUS>(B, grid, s);
    case GMQ_POLY_SUMSQ11: return batch_launch_rule64_family<GMQ_POLY_SUMSQ11>(B, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int batch_rule64_max_blocks(int fam, int dmax) {
  switch (fam) {
    case GMQ_OSCILLATORY: return batch_rule64_max_blocks_family<GMQ_OSCILLATORY>(dmax);
    case GMQ_PRODUCT_PEAK: return batch_rule64_max_blocks_family<GMQ_PRODUCT_PEAK>(dmax);
    case GMQ_CORNER_PEAK: return batch_rule64_max_blocks_family<GMQ_CORNER_PEAK>(dmax);
    case GMQ_GAUSSIAN: return batch_rule64_max_blocks_family<GMQ_GAUSSIAN>(dmax);
    case GMQ_C0: return batch_rule64_max_blocks_family<GMQ_C0>(dmax);
    case GMQ_DISCONTINUOUS: return batch_rule64_max_blocks_family<GMQ_DISCONTINUOUS>(dmax);
    case GMQ_POLY_SUMSQ11: return batch_rule64_max_blocks_family<GMQ_POLY_SUMSQ11>(dmax);
    default: return 1;
  }
}

int batch_rule_mixed_max_blocks(int fam, int dmax) {
  switch (fam) {
    case GMQ_OSCILLATORY: return batch_rule_mixed_max_blocks_family<GMQ_OSCILLATORY>(dmax);
    case GMQ_PRODUCT_PEAK: return batch_rule_mixed_max_blocks_family<GMQ_PRODUCT_PEAK>(dmax);
    case GMQ_CORNER_PEAK: return batch_rule_mixed_max_blocks_family<GMQ_CORNER_PEAK>(dmax);
    case GMQ_GAUSSIAN: return batch_rule_mixed_max_blocks_family<GMQ_GAUSSIAN>(dmax);
    case GMQ_C0: return batch_rule_mixed_max_blocks_family<GMQ_C0>(dmax);
    case GMQ_DISCONTINUOUS: return batch_rule_mixed_max_blocks_family<GMQ_DISCONTINUOUS>(dmax);
    default: return batch_rule_mixed_max_blocks_family<GMQ_POLY_SUMSQ11>(dmax);
  }
}

// ---- Gauss-Kronrod (7, 15) tables, computed on the host in FP64 ----------
// P_n(x) and P_n'(x) by the three-term recurrence.
void legendre_pd(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *p = 1.0;
    *dp = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// The n / 2 positive zeros of P_n (descending) by Newton from the usual
// cosine guesses cos(pi (i + 3/4) / (n + 1/2)), i = 0 .. n/2 - 1 (for odd n
// the zero at 0 is not among them); ws (if not null) the Gauss weights.
void gauss_positive(int n, double* xs, double* ws) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n / 2; ++i) {
    double x = std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre_pd(n, x, &p, &dp);
      const double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    double p, dp;
    legendre_pd(n, x, &p, &dp);
    xs[i] = x;
    if (ws) ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Dense solve with partial pivoting (n <= 8).
void solve_small(int n, double* a, double* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
    for (int k = 0; k < n; ++k) std::swap(a[c * n + k], a[piv * n + k]);
    std::swap(b[c], b[piv]);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c] / a[c * n + c];
      for (int k = 0; k < n; ++k) a[r * n + k] -= f * a[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int c = 0; c < n; ++c) b[c] /= a[c * n + c];
}

GkConst make_gk() {
  GkConst K;
  // positive G7 nodes (ascending) and weights; the centre separately
  double g[3], gw[3];
  gauss_positive(7, g, gw);
  std::sort(g, g + 3);
  for (int i = 0; i < 3; ++i) {
    double p, dp;
    legendre_pd(7, g[i], &p, &dp);
    gw[i] = 2.0 / ((1.0 - g[i] * g[i]) * dp * dp);
  }
  double p0, dp0;
  legendre_pd(7, 0.0, &p0, &dp0);
  const double gw0 = 2.0 / (dp0 * dp0);
  // Stieltjes polynomial E8 = sum_{m<=4} a_m P_{2m}, a_4 = 1, orthogonal to
  // P7 x^k (k odd; the even k vanish by parity): moments by a 16-point
  // Gauss rule (exact to degree 31 >= 8 + 7 + 7)
  double q[8], qw[8];
  gauss_positive(16, q, qw);
  auto moment = [&](int m2, int k) {
    double acc = 0.0;
    for (int i = 0; i < 8; ++i) {
      double pa, da, pb, db;
      legendre_pd(m2, q[i], &pa, &da);
      legendre_pd(7, q[i], &pb, &db);
      acc += 2.0 * qw[i] * pa * pb * std::pow(q[i], k);  // the integrand is even
    }
    return acc;
  };
  double M[16], rhs[4];
  const int ks[4] = {1, 3, 5, 7};
  for (int r = 0; r < 4; ++r) {
    for (int m = 0; m < 4; ++m) M[r * 4 + m] = moment(2 * m, ks[r]);
    rhs[r] = -moment(8, ks[r]);
  }
  solve_small(4, M, rhs);
  auto e8 = [&](double x) {
    double v = 0.0, p, dp;
    for (int m = 0; m < 4; ++m) {
      legendre_pd(2 * m, x, &p, &dp);
      v += rhs[m] * p;
    }
    legendre_pd(8, x, &p, &dp);
    return v + p;
  };
  // its positive zeros interlace the Gauss nodes: bisection in each gap
  const double edges[5] = {0.0, g[0], g[1], g[2], 1.0};
  double kz[4];
  for (int i = 0; i < 4; ++i) {
    double lo = edges[i], hi = edges[i + 1], flo = e8(lo);
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      const double fm = e8(mid);
      if ((fm > 0.0) == (flo > 0.0)) {
        lo = mid;
        flo = fm;
      } else {
        hi = mid;
      }
    }
    kz[i] = 0.5 * (lo + hi);
  }
  // the 7 positive nodes, alternating Kronrod-only and Gauss
  const double pos[7] = {kz[0], g[0], kz[1], g[1], kz[2], g[2], kz[3]};
  // K15 weights: exactness for P_0, P_2, ..., P_14 over the centre and the
  // 7 symmetric pairs
  double W[64], wb[8];
  const double dist[8] = {0.0, pos[0], pos[1], pos[2], pos[3], pos[4], pos[5], pos[6]};
  for (int r = 0; r < 8; ++r) {
    for (int j = 0; j < 8; ++j) {
      double p, dp;
      legendre_pd(2 * r, dist[j], &p, &dp);
      W[r * 8 + j] = (j == 0 ? 1.0 : 2.0) * p;
    }
    wb[r] = (r == 0) ? 2.0 : 0.0;
  }
  solve_small(8, W, wb);
  for (int i = 0; i < 7; ++i) {
    K.x[6 - i] = -pos[i];
    K.x[8 + i] = pos[i];
    K.wk[6 - i] = K.wk[8 + i] = wb[1 + i];
    const double gwi = (i % 2 == 1) ? gw[i / 2] : 0.0;
    K.wg[6 - i] = K.wg[8 + i] = gwi;
  }
  K.x[7] = 0.0;
  K.wk[7] = wb[0];
  K.wg[7] = gw0;
  for (int j = 0; j < 15; ++j) K.r[j] = 1.0 - K.wg[j] / K.wk[j];
  return K;
}

cudaError_t launch_rule_gk(int fam, const GkArgs& G, cudaStream_t s) {
  switch (fam) {
    case GMQ_OSCILLATORY: return launch_rule_gk_family<GMQ_OSCILLATORY>(G, s);
    case GMQ_PRODUCT_PEAK: return launch_rule_gk_family<GMQ_PRODUCT_PEAK>(G, s);
    case GMQ_CORNER_PEAK: return launch_rule_gk_family<GMQ_CORNER_PEAK>(G, s);
    case GMQ_GAUSSIAN: return launch_rule_gk_family<GMQ_GAUSSIAN>(G, s);
    case GMQ_C0: return launch_rule_gk_family<GMQ_C0>(G, s);
    case GMQ_DISCONTINUOUS: return launch_rule_gk_family<GMQ_DISCONTINUOUS>(G, s);
    case GMQ_POLY_SUMSQ11: return launch_rule_gk_family<GMQ_POLY_SUMSQ11>(G, s);
    default: return cudaErrorInvalidValue;
  }
}

// Two CUDA events released when the holder goes out of scope.
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Name of the last CUDA error a call of this thread turned into a status.
thread_local const char* g_last_cuda_error = "cudaSuccess";

gmq_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorName(e);
  if (e == cudaErrorMemoryAllocation) return GMQ_ERR_OOM;
  if (e == cudaErrorNotSupported) return GMQ_ERR_INVALID;
  return GMQ_ERR_CUDA;
}

#define GMQ_CK(expr)                          \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// Pool memory for an integration: the caller's pool or library memory that
// grows on demand.
gmq_status ensure_pool(gmq_context* ctx, size_t need, char** base) {
  if (ctx->ext) {
    if (ctx->ext_bytes < need) return GMQ_ERR_OOM;
    *base = ctx->ext;
    return GMQ_OK;
  }
  if (ctx->own_bytes < need) {
    if (ctx->own) {
      cudaFree(ctx->own);
      ctx->own = nullptr;
      ctx->own_bytes = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return GMQ_ERR_OOM;
    }
    ctx->own = (char*)p;
    ctx->own_bytes = need;
  }
  *base = ctx->own;
  return GMQ_OK;
}

// Kernel timing: events around each launch, collected after the stream wait.
enum { kKRule = 0, kKSum = 1, kKClassify = 2, kKSplit = 3, kKPartition = 4 };

inline void prof_begin(gmq_context* c, int k) {
  if (c->prof_on) cudaEventRecord(c->ev[k][0], c->stream);
}

inline void prof_end(gmq_context* c, int k, int64_t regions) {
  if (!c->prof_on) return;
  cudaEventRecord(c->ev[k][1], c->stream);
  c->pending[k] = true;
  c->pend_regions[k] = regions;
}

void prof_collect(gmq_context* c) {
  if (!c->prof_on) return;
  for (int k = 0; k < 5; ++k) {
    if (!c->pending[k]) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[k][0], c->ev[k][1]) == cudaSuccess) {
      c->stats[k].ms += ms;
      c->stats[k].launches += 1;
      c->stats[k].regions += c->pend_regions[k];
    } else {
      cudaGetLastError();
    }
    c->pending[k] = false;
  }
}

// Scratch of the step-level calls: per-tile arrays for n regions, a flag
// array, and a device status.
struct Scratch {
  int* cnt;
  long long* off;
  double* ba;
  double* bb;
  uint8_t* flags;
  DevStatus* st;
  double* out;
};

gmq_status ensure_scratch(gmq_context* ctx, int64_t n, Scratch* S) {
  const int64_t nb = std::max<int64_t>(1, (n + kTile - 1) / kTile);
  size_t p = 0;
  const size_t o_cnt = p; p += align256(sizeof(int) * nb);
  const size_t o_off = p; p += align256(sizeof(long long) * nb);
  const size_t o_ba = p; p += align256(sizeof(double) * nb);
  const size_t o_bb = p; p += align256(sizeof(double) * nb);
  const size_t o_fl = p; p += align256((size_t)std::max<int64_t>(n, 1));
  const size_t o_st = p; p += align256(sizeof(DevStatus));
  const size_t o_out = p; p += 256;
  if (ctx->scratch_bytes < p) {
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    void* q = nullptr;
    if (cudaMalloc(&q, p) != cudaSuccess) {
      cudaGetLastError();
      return GMQ_ERR_OOM;
    }
    ctx->scratch = (char*)q;
    ctx->scratch_bytes = p;
  }
  char* b = ctx->scratch;
  S->cnt = (int*)(b + o_cnt);
  S->off = (long long*)(b + o_off);
  S->ba = (double*)(b + o_ba);
  S->bb = (double*)(b + o_bb);
  S->flags = (uint8_t*)(b + o_fl);
  S->st = (DevStatus*)(b + o_st);
  S->out = (double*)(b + o_out);
  return GMQ_OK;
}

}  // namespace

const GkConst& gmq::gk_const() {
  static const GkConst K = make_gk();
  return K;
}

namespace {

// The context's device copy of the Gauss-Kronrod tables (made on first use).
gmq_status ensure_gk(gmq_context* ctx) {
  if (ctx->gk_dev) return GMQ_OK;
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(GkConst)) != cudaSuccess) {
    cudaGetLastError();
    return GMQ_ERR_OOM;
  }
  const cudaError_t e = cudaMemcpy(q, &gk_const(), sizeof(GkConst), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(q);
    return cuda_fail(e);
  }
  ctx->gk_dev = (GkConst*)q;
  return GMQ_OK;
}

}  // namespace

extern "C" {

const char* gmq_status_string(gmq_status s) {
  switch (s) {
    case GMQ_OK: return "converged";
    case GMQ_CAP_REACHED: return "region cap reached";
    case GMQ_MAX_ITERS: return "iteration limit reached";
    case GMQ_ROUNDOFF_LIMIT: return "all regions retired before the tolerance was met";
    case GMQ_ERR_INVALID: return "invalid argument";
    case GMQ_ERR_OOM: return "out of device memory";
    case GMQ_ERR_CUDA: return "CUDA error";
    case GMQ_ERR_NONFINITE: return "non-finite integrand value";
    case GMQ_ERR_TIMEOUT: return "device wait timed out";
    case GMQ_ERR_TOO_LARGE: return "input longer than the fixed scratch allows";
  }
  return "unknown status";
}

const char* gmq_last_cuda_error(void) { return g_last_cuda_error; }

gmq_status gmq_create(gmq_context** out, int device, size_t pool_bytes_hint) {
  if (!out) return GMQ_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return GMQ_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return GMQ_ERR_INVALID;
  DeviceGuard g(device);
  if (!g.ok) return GMQ_ERR_CUDA;
  gmq_context* ctx = new (std::nothrow) gmq_context();
  if (!ctx) return GMQ_ERR_OOM;
  ctx->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return GMQ_ERR_CUDA;
  }
  ctx->sm_count = prop.multiProcessorCount;
  // pinned status buffer: one sweep's DevStatus, or a batch's BatchState
  constexpr size_t kHostStatusBytes =
      sizeof(DevStatus) > sizeof(BatchState) ? sizeof(DevStatus) : sizeof(BatchState);
  if (cudaHostAlloc((void**)&ctx->h_status, kHostStatusBytes, cudaHostAllocDefault) != cudaSuccess) {
    delete ctx;
    return GMQ_ERR_CUDA;
  }
  if (pool_bytes_hint > 0) {
    char* base = nullptr;
    gmq_status st = ensure_pool(ctx, pool_bytes_hint, &base);
    if (st != GMQ_OK) {
      cudaFreeHost(ctx->h_status);
      delete ctx;
      return st;
    }
  }
  *out = ctx;
  return GMQ_OK;
}

gmq_status gmq_destroy(gmq_context* ctx) {
  if (!ctx) return GMQ_ERR_INVALID;
  {
    DeviceGuard g(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->own) cudaFree(ctx->own);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->gscratch) cudaFree(ctx->gscratch);
    if (ctx->gk_dev) cudaFree(ctx->gk_dev);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->ev_made)
      for (int k = 0; k < 5; ++k)
        for (int j = 0; j < 2; ++j) cudaEventDestroy(ctx->ev[k][j]);
  }
  delete ctx;
  return GMQ_OK;
}

gmq_status gmq_set_stream(gmq_context* ctx, void* cuda_stream) {
  if (!ctx) return GMQ_ERR_INVALID;
  ctx->stream = (cudaStream_t)cuda_stream;
  return GMQ_OK;
}

gmq_status gmq_set_pool(gmq_context* ctx, void* dev_ptr, size_t bytes) {
  if (!ctx) return GMQ_ERR_INVALID;
  if (dev_ptr && ((uintptr_t)dev_ptr & 255u)) return GMQ_ERR_INVALID;
  ctx->ext = (char*)dev_ptr;
  ctx->ext_bytes = dev_ptr ? bytes : 0;
  return GMQ_OK;
}

gmq_status gmq_set_eval_mode(gmq_context* ctx, int32_t mode) {
  if (!ctx || (mode != GMQ_EVAL_SEPARABLE && mode != GMQ_EVAL_NODEWISE)) return GMQ_ERR_INVALID;
  ctx->eval_mode = mode;
  return GMQ_OK;
}

gmq_status gmq_pool_bytes(int32_t dim, int64_t max_regions, int32_t flags, size_t* bytes) {
  if (!bytes || dim < 1 || dim > GMQ_MAX_DIM || max_regions < 1 || max_regions > kMaxRegions ||
      (flags & ~GMQ_KEEP_PARTITION))
    return GMQ_ERR_INVALID;
  *bytes = pool_layout(dim, max_regions, flags).total;
  return GMQ_OK;
}

gmq_status gmq_default_options(gmq_options* opt) {
  if (!opt) return GMQ_ERR_INVALID;
  std::memset(opt, 0, sizeof(*opt));
  opt->rel_tol = 1e-6;
  opt->abs_tol = 1e-16;
  opt->max_regions = (int64_t)1 << 22;
  opt->max_iters = 1000;
  opt->precision = GMQ_FP64;
  opt->classifier = GMQ_VOLUME_SHARE;
  opt->rule = GMQ_RULE_GENZ_MALIK;
  return GMQ_OK;
}

gmq_status gmq_launch_count(gmq_context* ctx, int64_t* count) {
  if (!ctx || !count) return GMQ_ERR_INVALID;
  *count = ctx->launches;
  return GMQ_OK;
}

gmq_status gmq_last_trace(gmq_context* ctx, gmq_sweep* out, int32_t max, int32_t* count) {
  if (!ctx || !count || max < 0 || (max > 0 && !out)) return GMQ_ERR_INVALID;
  *count = (int32_t)ctx->trace.size();
  const int32_t m = std::min<int32_t>(max, *count);
  for (int32_t i = 0; i < m; ++i) out[i] = ctx->trace[i];
  return GMQ_OK;
}

gmq_status gmq_seed_genz(uint64_t seed, int32_t family, int32_t dim, double target_sum,
                         double* a_out, double* u_out) {
  if (dim < 1 || dim > 255 || family < 0 || family > 255 || !a_out || !u_out) return GMQ_ERR_INVALID;
  // SplitMix64 (Steele, Lea & Flood 2014)
  uint64_t state = (seed << 16) ^ ((uint64_t)family << 8) ^ (uint64_t)dim;
  auto next = [&state]() -> double {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  double tot = 0.0;
  for (int j = 0; j < dim; ++j) {
    a_out[j] = next();
    tot = tot + a_out[j];
  }
  for (int j = 0; j < dim; ++j) u_out[j] = next();
  const double scale = target_sum / tot;
  for (int j = 0; j < dim; ++j) a_out[j] = a_out[j] * scale;
  return GMQ_OK;
}

gmq_status gmq_integrate(gmq_context* ctx, const gmq_problem* prob, const gmq_options* opt,
                         gmq_result* out) {
  NvtxRange range("gmq_integrate");
  if (!ctx || !opt || !out) return GMQ_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  ctx->trace.clear();
  gmq_status vs = validate_problem(prob);
  if (vs != GMQ_OK) return out->status = vs, vs;
  const int d = prob->dim;
  const int64_t cap = opt->max_regions;
  if (!(opt->rel_tol >= 0.0) || !(opt->abs_tol >= 0.0) || cap < 1 || cap > kMaxRegions ||
      opt->init_splits < 0 || opt->max_iters < 0 || (opt->flags & ~GMQ_KEEP_PARTITION) ||
      (opt->precision != GMQ_FP64 && opt->precision != GMQ_MIXED) ||
      (opt->classifier != GMQ_VOLUME_SHARE && opt->classifier != GMQ_LOCAL_REL) ||
      (opt->lanes != 0 && opt->lanes != 1 && opt->lanes != 4 && opt->lanes != 32 &&
       opt->lanes != 128) ||
      (opt->lanes == 128 && opt->precision != GMQ_FP64) ||
      (opt->rule != GMQ_RULE_GENZ_MALIK && opt->rule != GMQ_RULE_GAUSS_KRONROD) ||
      (opt->rule == GMQ_RULE_GAUSS_KRONROD &&
       (opt->precision != GMQ_FP64 || d > GMQ_GK_MAX_DIM ||
        opt->estimator != GMQ_EST_EMBEDDED)) ||
      (opt->estimator != GMQ_EST_EMBEDDED && opt->estimator != GMQ_EST_NULL_RULES))
    return out->status = GMQ_ERR_INVALID, GMQ_ERR_INVALID;
  const bool gk = opt->rule == GMQ_RULE_GAUSS_KRONROD;
  const int s = opt->init_splits > 0 ? opt->init_splits : auto_splits(d, cap);
  int64_t n = 1;
  for (int k = 0; k < d; ++k) {
    n *= s;
    if (n > cap) return out->status = GMQ_ERR_INVALID, GMQ_ERR_INVALID;
  }
  const int max_iters = opt->max_iters > 0 ? opt->max_iters : 1000;

  DeviceGuard g(ctx->device);
  if (!g.ok) return out->status = GMQ_ERR_CUDA, GMQ_ERR_CUDA;
  const bool keep = (opt->flags & GMQ_KEEP_PARTITION) != 0;
  ctx->part_count = -1;
  const PoolLayout L = pool_layout(d, cap, opt->flags);
  char* base = nullptr;
  gmq_status ps = ensure_pool(ctx, L.total, &base);
  if (ps != GMQ_OK) return out->status = ps, ps;

  double* cA = (double*)(base + L.cA);
  double* hA = (double*)(base + L.hA);
  double* cB = (double*)(base + L.cB);
  double* hB = (double*)(base + L.hB);
  DevStatus* st = (DevStatus*)(base + L.st);
  cudaStream_t strm = ctx->stream;

  const FamParams P = fam_params(prob);
  const RuleConst R = rule_const(d, prob->lo, prob->hi, opt->estimator);
  int64_t nodes_per_region = R.nodes;
  if (gk) {
    gmq_status gs = ensure_gk(ctx);
    if (gs != GMQ_OK) return out->status = gs, gs;
    nodes_per_region = 1;
    for (int k = 0; k < d; ++k) nodes_per_region *= 15;
  }

  // initial uniform partition
  PartArgs PA;
  std::memset(&PA, 0, sizeof(PA));
  PA.d = d;
  PA.s = s;
  PA.n = n;
  for (int k = 0; k < d; ++k) {
    const double lo = prob->lo ? prob->lo[k] : 0.0, hi = prob->hi ? prob->hi[k] : 1.0;
    PA.lo[k] = lo;
    PA.h[k] = (hi - lo) / (2.0 * (double)s);
  }
  PA.c_out = cA;
  PA.h_out = hA;
  PA.ld = L.ld;
  GMQ_CK(cudaMemsetAsync(st, 0, sizeof(DevStatus), strm));
  prof_begin(ctx, kKPartition);
  GMQ_CK(launch_partition(PA, strm));
  prof_end(ctx, kKPartition, n);
  ctx->launches += 1;

  gmq_status status = GMQ_OK;
  int iters = 0;
  for (;;) {
    char sweep_name[64];
    std::snprintf(sweep_name, sizeof(sweep_name), "sweep %d: %lld regions", iters + 1,
                  (long long)n);
    NvtxRange sweep_range(sweep_name);
    const int T = choose_lanes(opt->lanes, n, d, ctx->sm_count, opt->precision);
    RuleArgs A;
    A.c = cA;
    A.h = hA;
    A.ld = L.ld;
    A.n = n;
    A.i7 = (double*)(base + L.i7);
    A.err = (double*)(base + L.err);
    A.volfrac = (double*)(base + L.vf);
    A.axis = (uint8_t*)(base + L.axis);
    A.P = P;
    A.R = R;
    A.nodewise = ctx->eval_mode == GMQ_EVAL_NODEWISE ? 1 : 0;
    prof_begin(ctx, kKRule);
    if (gk) {
      GkArgs GA;
      GA.A = A;
      GA.K = ctx->gk_dev;
      GMQ_CK(launch_rule_gk(prob->family, GA, strm));
    } else {
      GMQ_CK(launch_rule(prob->family, opt->precision, T, A, strm));
    }
    prof_end(ctx, kKRule, n);

    SweepArgs S;
    std::memset(&S, 0, sizeof(S));
    S.n = n;
    S.d = d;
    S.classifier = opt->classifier;
    S.rel_tol = opt->rel_tol;
    S.abs_tol = opt->abs_tol;
    S.cap = cap;
    S.c = cA;
    S.h = hA;
    S.ld = L.ld;
    S.c_out = cB;
    S.h_out = hB;
    S.ld_out = L.ld;
    S.i7 = A.i7;
    S.err = A.err;
    S.volfrac = A.volfrac;
    S.axis = A.axis;
    S.flags = (uint8_t*)(base + L.flags);
    S.blk_count = (int*)(base + L.cnt);
    S.blk_off = (long long*)(base + L.off);
    S.blk_a = (double*)(base + L.ba);
    S.blk_b = (double*)(base + L.bb);
    S.budget_ptr = &st->budget;
    S.guard = opt->precision == GMQ_MIXED ? kGuardMixed : kGuardFp64;
    S.last_sweep = (iters + 1 >= max_iters) ? 1 : 0;
    S.keep = keep ? 1 : 0;
    S.c_leaf = keep ? (double*)(base + L.cL) : nullptr;
    S.h_leaf = keep ? (double*)(base + L.hL) : nullptr;
    S.ld_leaf = L.ld;
    S.leaf_cap = cap;
    S.st = st;
    prof_begin(ctx, kKSum);
    GMQ_CK(launch_sum_status(S, strm));
    prof_end(ctx, kKSum, n);
    prof_begin(ctx, kKClassify);
    GMQ_CK(launch_classify(S, strm));
    prof_end(ctx, kKClassify, n);
    prof_begin(ctx, kKSplit);
    GMQ_CK(launch_split(S, strm));
    prof_end(ctx, kKSplit, n);
    ctx->launches += 4;
    GMQ_CK(cudaMemcpyAsync(ctx->h_status, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, strm));
    GMQ_CK(cudaStreamSynchronize(strm));
    prof_collect(ctx);
    const DevStatus h = *ctx->h_status;

    ++iters;
    out->regions_evaluated += n;
    out->function_evals += n * nodes_per_region;
    out->final_active = n;
    out->integral = h.I;
    out->error = h.E;
    gmq_sweep rec;
    rec.n = n;
    rec.I = h.I;
    rec.E = h.E;
    rec.budget = h.budget;
    // the loop classifies only when it neither stopped nor hit the sweep
    // limit; the classify kernel ran regardless, so an unclassified record
    // carries the retired sums of the previous sweep
    const bool classified = !(h.flags & (kConverged | kNonfinite)) && iters < max_iters;
    rec.n_split = classified ? h.n_split : -1;
    rec.I_ret = classified ? h.I_ret : (ctx->trace.empty() ? 0.0 : ctx->trace.back().I_ret);
    rec.E_ret = classified ? h.E_ret : (ctx->trace.empty() ? 0.0 : ctx->trace.back().E_ret);
    ctx->trace.push_back(rec);

    if (h.flags & kNonfinite) {
      status = GMQ_ERR_NONFINITE;
      break;
    }
    if (h.flags & kConverged) {
      status = GMQ_OK;
      break;
    }
    if (iters >= max_iters) {
      status = GMQ_MAX_ITERS;
      break;
    }
    if (h.flags & kAllRetired) {
      status = GMQ_ROUNDOFF_LIMIT;
      break;
    }
    if (h.flags & (kCapExceeded | kLeafOverflow)) {
      status = GMQ_CAP_REACHED;
      break;
    }
    n = 2 * h.n_split;
    std::swap(cA, cB);
    std::swap(hA, hB);
  }
  out->iterations = iters;
  out->status = status;
  // final partition: the leaves recorded so far plus the last sweep's list
  if (keep && status != GMQ_ERR_NONFINITE && !(ctx->h_status->flags & kLeafOverflow)) {
    const long long base_leaves = ctx->h_status->n_leaves;
    if (base_leaves + n <= cap) {
      double* cL = (double*)(base + L.cL);
      double* hL = (double*)(base + L.hL);
      const size_t pitch = sizeof(double) * (size_t)L.ld;
      GMQ_CK(cudaMemcpy2DAsync(cL + base_leaves, pitch, cA, pitch, sizeof(double) * (size_t)n, d,
                               cudaMemcpyDeviceToDevice, strm));
      GMQ_CK(cudaMemcpy2DAsync(hL + base_leaves, pitch, hA, pitch, sizeof(double) * (size_t)n, d,
                               cudaMemcpyDeviceToDevice, strm));
      GMQ_CK(cudaStreamSynchronize(strm));
      ctx->part_count = base_leaves + n;
      ctx->part_d = d;
      ctx->part_ld = L.ld;
      ctx->part_c = cL;
      ctx->part_h = hL;
    }
  }
  return status;
}

gmq_status gmq_eval_rule(gmq_context* ctx, const gmq_problem* prob, int32_t precision,
                         int32_t lanes, int32_t estimator, int64_t n, const double* d_center,
                         const double* d_halfw,
                         int64_t ld, double* d_integral, double* d_error, double* d_volfrac,
                         uint8_t* d_axis) {
  if (!ctx) return GMQ_ERR_INVALID;
  gmq_status vs = validate_problem(prob);
  if (vs != GMQ_OK) return vs;
  if (n < 0 || ld < n || (n > 0 && (!d_center || !d_halfw || !d_integral || !d_error || !d_axis)))
    return GMQ_ERR_INVALID;
  if (precision != GMQ_FP64 && precision != GMQ_MIXED) return GMQ_ERR_INVALID;
  if (lanes != 0 && lanes != 1 && lanes != 4 && lanes != 32 && lanes != 128)
    return GMQ_ERR_INVALID;
  if (lanes == 128 && precision != GMQ_FP64) return GMQ_ERR_INVALID;
  if (estimator != GMQ_EST_EMBEDDED && estimator != GMQ_EST_NULL_RULES) return GMQ_ERR_INVALID;
  if (n == 0) return GMQ_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  RuleArgs A;
  A.c = d_center;
  A.h = d_halfw;
  A.ld = ld;
  A.n = n;
  A.i7 = d_integral;
  A.err = d_error;
  A.volfrac = d_volfrac;
  A.axis = d_axis;
  A.P = fam_params(prob);
  A.R = rule_const(prob->dim, prob->lo, prob->hi, estimator);
  A.nodewise = ctx->eval_mode == GMQ_EVAL_NODEWISE ? 1 : 0;
  const int T = choose_lanes(lanes, n, prob->dim, ctx->sm_count, precision);
  prof_begin(ctx, kKRule);
  GMQ_CK(launch_rule(prob->family, precision, T, A, ctx->stream));
  prof_end(ctx, kKRule, n);
  ctx->launches += 1;
  GMQ_CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  return GMQ_OK;
}

gmq_status gmq_eval_rule_gk(gmq_context* ctx, const gmq_problem* prob, int64_t n,
                            const double* d_center, const double* d_halfw, int64_t ld,
                            double* d_integral, double* d_error, double* d_volfrac,
                            uint8_t* d_axis) {
  if (!ctx) return GMQ_ERR_INVALID;
  gmq_status vs = validate_problem(prob);
  if (vs != GMQ_OK) return vs;
  if (prob->dim > GMQ_GK_MAX_DIM) return GMQ_ERR_INVALID;
  if (n < 0 || ld < n || (n > 0 && (!d_center || !d_halfw || !d_integral || !d_error || !d_axis)))
    return GMQ_ERR_INVALID;
  if (n == 0) return GMQ_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  gmq_status gs = ensure_gk(ctx);
  if (gs != GMQ_OK) return gs;
  GkArgs G;
  G.A.c = d_center;
  G.A.h = d_halfw;
  G.A.ld = ld;
  G.A.n = n;
  G.A.i7 = d_integral;
  G.A.err = d_error;
  G.A.volfrac = d_volfrac;
  G.A.axis = d_axis;
  G.A.P = fam_params(prob);
  G.A.R = rule_const(prob->dim, prob->lo, prob->hi);
  G.A.nodewise = 0;
  G.K = ctx->gk_dev;
  prof_begin(ctx, kKRule);
  GMQ_CK(launch_rule_gk(prob->family, G, ctx->stream));
  prof_end(ctx, kKRule, n);
  ctx->launches += 1;
  GMQ_CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  return GMQ_OK;
}

}  // extern "C"

namespace {
__global__ void k_math_exp(int64_t n, const double* x, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = gm_exp(x[i]);
}
__global__ void k_math_rcp(int64_t n, const double* x, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = gm_rcp(x[i]);
}
__global__ void k_math_cos(int64_t n, const double* x, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = gm_cos(x[i]);
}
}  // namespace

extern "C" {

gmq_status gmq_math_exp(gmq_context* ctx, int64_t n, const double* d_x, double* d_y) {
  if (!ctx || n < 0 || (n > 0 && (!d_x || !d_y))) return GMQ_ERR_INVALID;
  if (n == 0) return GMQ_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  k_math_exp<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, d_x, d_y);
  GMQ_CK(cudaGetLastError());
  ctx->launches += 1;
  GMQ_CK(cudaStreamSynchronize(ctx->stream));
  return GMQ_OK;
}

gmq_status gmq_math_rcp(gmq_context* ctx, int64_t n, const double* d_x, double* d_y) {
  if (!ctx || n < 0 || (n > 0 && (!d_x || !d_y))) return GMQ_ERR_INVALID;
  if (n == 0) return GMQ_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  k_math_rcp<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, d_x, d_y);
  GMQ_CK(cudaGetLastError());
  ctx->launches += 1;
  GMQ_CK(cudaStreamSynchronize(ctx->stream));
  return GMQ_OK;
}

gmq_status gmq_math_cos(gmq_context* ctx, int64_t n, const double* d_x, double* d_y) {
  if (!ctx || n < 0 || (n > 0 && (!d_x || !d_y))) return GMQ_ERR_INVALID;
  if (n == 0) return GMQ_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  k_math_cos<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, d_x, d_y);
  GMQ_CK(cudaGetLastError());
  ctx->launches += 1;
  GMQ_CK(cudaStreamSynchronize(ctx->stream));
  return GMQ_OK;
}

gmq_status gmq_null_rule_table(int32_t dim, double* out) {
  if (!out || dim < 1 || dim > GMQ_MAX_DIM) return GMQ_ERR_INVALID;
  const RuleConst R = rule_const(dim, nullptr, nullptr, GMQ_EST_NULL_RULES);
  for (int k = 0; k < 20; ++k) out[k] = R.nw[k];
  return GMQ_OK;
}

gmq_status gmq_gk_table(double* out) {
  if (!out) return GMQ_ERR_INVALID;
  const GkConst& K = gk_const();
  for (int j = 0; j < 15; ++j) {
    out[j] = K.x[j];
    out[15 + j] = K.wk[j];
    out[30 + j] = K.wg[j];
  }
  return GMQ_OK;
}

gmq_status gmq_classify_split(gmq_context* ctx, int32_t dim, int64_t n, const double* d_center,
                              const double* d_halfw, int64_t ld, const double* d_integral,
                              const double* d_error, const double* d_volfrac,
                              const uint8_t* d_axis, double budget, double rel_tol,
                              int32_t classifier, double* d_center_out, double* d_halfw_out,
                              int64_t ld_out, int64_t cap_out, uint8_t* d_flags,
                              int64_t* n_split, double* retired_integral,
                              double* retired_error) {
  if (!ctx || !n_split || !retired_integral || !retired_error) return GMQ_ERR_INVALID;
  if (dim < 1 || dim > GMQ_MAX_DIM || n < 0 || n > kMaxRegions || ld < n || cap_out < 0 ||
      ld_out < cap_out)
    return GMQ_ERR_INVALID;
  if (classifier != GMQ_VOLUME_SHARE && classifier != GMQ_LOCAL_REL) return GMQ_ERR_INVALID;
  if (n > 0 && (!d_center || !d_halfw || !d_integral || !d_error || !d_axis ||
                (classifier == GMQ_VOLUME_SHARE && !d_volfrac)))
    return GMQ_ERR_INVALID;
  if (cap_out > 0 && (!d_center_out || !d_halfw_out)) return GMQ_ERR_INVALID;
  *n_split = 0;
  *retired_integral = 0.0;
  *retired_error = 0.0;
  if (n == 0) return GMQ_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  Scratch X;
  gmq_status ss = ensure_scratch(ctx, n, &X);
  if (ss != GMQ_OK) return ss;
  SweepArgs S;
  std::memset(&S, 0, sizeof(S));
  S.n = n;
  S.d = dim;
  S.classifier = classifier;
  S.rel_tol = rel_tol;
  S.cap = cap_out;
  S.c = d_center;
  S.h = d_halfw;
  S.ld = ld;
  S.c_out = d_center_out;
  S.h_out = d_halfw_out;
  S.ld_out = ld_out;
  S.i7 = d_integral;
  S.err = d_error;
  S.volfrac = d_volfrac;
  S.axis = d_axis;
  S.flags = d_flags ? d_flags : X.flags;
  S.blk_count = X.cnt;
  S.blk_off = X.off;
  S.blk_a = X.ba;
  S.blk_b = X.bb;
  S.budget_ptr = nullptr;
  S.budget_val = budget;
  S.guard = kGuardFp64;
  S.st = X.st;
  cudaStream_t strm = ctx->stream;
  GMQ_CK(cudaMemsetAsync(X.st, 0, sizeof(DevStatus), strm));
  prof_begin(ctx, kKClassify);
  GMQ_CK(launch_classify(S, strm));
  prof_end(ctx, kKClassify, n);
  prof_begin(ctx, kKSplit);
  GMQ_CK(launch_split(S, strm));
  prof_end(ctx, kKSplit, n);
  ctx->launches += 2;
  GMQ_CK(cudaMemcpyAsync(ctx->h_status, X.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, strm));
  GMQ_CK(cudaStreamSynchronize(strm));
  prof_collect(ctx);
  const DevStatus h = *ctx->h_status;
  *n_split = h.n_split;
  *retired_integral = h.ret_i;
  *retired_error = h.ret_e;
  if (h.flags & kCapExceeded) return GMQ_CAP_REACHED;
  return GMQ_OK;
}

gmq_status gmq_tree_sum(gmq_context* ctx, int64_t n, const double* d_v, double* sum) {
  if (!ctx || !sum || n < 0 || n > kMaxRegions || (n > 0 && !d_v)) return GMQ_ERR_INVALID;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  Scratch X;
  gmq_status ss = ensure_scratch(ctx, n, &X);
  if (ss != GMQ_OK) return ss;
  cudaStream_t strm = ctx->stream;
  GMQ_CK(cudaMemsetAsync(X.st, 0, sizeof(DevStatus), strm));
  prof_begin(ctx, kKSum);
  GMQ_CK(launch_tree_sum(d_v, n, X.ba, X.st, X.out, strm));
  prof_end(ctx, kKSum, n);
  ctx->launches += 1;
  GMQ_CK(cudaMemcpyAsync(&ctx->h_status->I, X.out, sizeof(double), cudaMemcpyDeviceToHost, strm));
  GMQ_CK(cudaStreamSynchronize(strm));
  prof_collect(ctx);
  *sum = ctx->h_status->I;
  return GMQ_OK;
}

gmq_status gmq_partition(gmq_context* ctx, int32_t dim, const double* lo, const double* hi,
                         int32_t s, double* d_center, double* d_halfw, int64_t ld) {
  if (!ctx || dim < 1 || dim > GMQ_MAX_DIM || s < 1 || !d_center || !d_halfw)
    return GMQ_ERR_INVALID;
  int64_t n = 1;
  for (int k = 0; k < dim; ++k) {
    n *= s;
    if (n > kMaxRegions) return GMQ_ERR_INVALID;
  }
  if (ld < n) return GMQ_ERR_INVALID;
  PartArgs PA;
  std::memset(&PA, 0, sizeof(PA));
  PA.d = dim;
  PA.s = s;
  PA.n = n;
  for (int k = 0; k < dim; ++k) {
    const double l = lo ? lo[k] : 0.0, h = hi ? hi[k] : 1.0;
    if (!std::isfinite(l) || !std::isfinite(h) || !(h > l)) return GMQ_ERR_INVALID;
    PA.lo[k] = l;
    PA.h[k] = (h - l) / (2.0 * (double)s);
  }
  PA.c_out = d_center;
  PA.h_out = d_halfw;
  PA.ld = ld;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  prof_begin(ctx, kKPartition);
  GMQ_CK(launch_partition(PA, ctx->stream));
  prof_end(ctx, kKPartition, n);
  ctx->launches += 1;
  GMQ_CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  return GMQ_OK;
}

gmq_status gmq_probe_fp_rate(gmq_context* ctx, int32_t precision, int32_t op, int64_t iters,
                             double* lane_ops_per_s, double* ms) {
  if (!ctx || !lane_ops_per_s || !ms || iters < 1 || iters > ((int64_t)1 << 32) ||
      (precision != GMQ_FP64 && precision != GMQ_MIXED) || op < 0 || op > 2)
    return GMQ_ERR_INVALID;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  const int blocks = ctx->sm_count * 8;  // 64 warps per SM
  const size_t sink = sizeof(double) * (size_t)blocks * kProbeBlock;
  if (ctx->gscratch_bytes < sink) {
    if (ctx->gscratch) cudaFree(ctx->gscratch);
    ctx->gscratch = nullptr;
    ctx->gscratch_bytes = 0;
    void* q = nullptr;
    if (cudaMalloc(&q, sink) != cudaSuccess) {
      cudaGetLastError();
      return GMQ_ERR_OOM;
    }
    ctx->gscratch = (char*)q;
    ctx->gscratch_bytes = sink;
  }
  EventPair ev;
  GMQ_CK(cudaEventCreate(&ev.a));
  GMQ_CK(cudaEventCreate(&ev.b));
  const int fp64 = precision == GMQ_FP64 ? 1 : 0;
  GMQ_CK(cudaEventRecord(ev.a, ctx->stream));
  GMQ_CK(launch_fma_probe(fp64, op, blocks, iters, ctx->gscratch, ctx->stream));
  GMQ_CK(cudaEventRecord(ev.b, ctx->stream));
  ctx->launches += 1;
  GMQ_CK(cudaEventSynchronize(ev.b));
  float t = 0.f;
  GMQ_CK(cudaEventElapsedTime(&t, ev.a, ev.b));
  *ms = (double)t;
  *lane_ops_per_s = t > 0.f ? (double)fma_probe_lane_fmas(blocks, iters) / ((double)t * 1e-3) : 0.0;
  return GMQ_OK;
}

gmq_status gmq_profile_enable(gmq_context* ctx, int32_t on) {
  if (!ctx) return GMQ_ERR_INVALID;
  if (on && !ctx->ev_made) {
    DeviceGuard g(ctx->device);
    for (int k = 0; k < 5; ++k)
      for (int j = 0; j < 2; ++j)
        if (cudaEventCreate(&ctx->ev[k][j]) != cudaSuccess) return GMQ_ERR_CUDA;
    ctx->ev_made = true;
  }
  ctx->prof_on = on != 0;
  return GMQ_OK;
}

gmq_status gmq_profile_reset(gmq_context* ctx) {
  if (!ctx) return GMQ_ERR_INVALID;
  for (int k = 0; k < 5; ++k) {
    ctx->stats[k] = gmq_kernel_stats{0, 0, 0.0};
    ctx->pending[k] = false;
  }
  return GMQ_OK;
}

gmq_status gmq_profile_read(gmq_context* ctx, int32_t kernel, gmq_kernel_stats* out) {
  if (!ctx || !out || kernel < 0 || kernel > 4) return GMQ_ERR_INVALID;
  *out = ctx->stats[kernel];
  return GMQ_OK;
}


gmq_status gmq_partition_copy(gmq_context* ctx, double* d_center, double* d_halfw, int64_t ld,
                              int64_t max, int64_t* count) {
  if (!ctx || !count || max < 0) return GMQ_ERR_INVALID;
  *count = ctx->part_count;
  if (ctx->part_count < 0) return GMQ_OK;
  const int64_t m = std::min<int64_t>(max, ctx->part_count);
  if (m == 0) return GMQ_OK;
  if (!d_center || !d_halfw || ld < m) return GMQ_ERR_INVALID;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  const size_t spitch = sizeof(double) * (size_t)ctx->part_ld, dpitch = sizeof(double) * (size_t)ld;
  GMQ_CK(cudaMemcpy2DAsync(d_center, dpitch, ctx->part_c, spitch, sizeof(double) * (size_t)m,
                           ctx->part_d, cudaMemcpyDeviceToDevice, ctx->stream));
  GMQ_CK(cudaMemcpy2DAsync(d_halfw, dpitch, ctx->part_h, spitch, sizeof(double) * (size_t)m,
                           ctx->part_d, cudaMemcpyDeviceToDevice, ctx->stream));
  GMQ_CK(cudaStreamSynchronize(ctx->stream));
  return GMQ_OK;
}

gmq_status gmq_last_batch_info(gmq_context* ctx, gmq_batch_info* info) {
  if (!ctx || !info) return GMQ_ERR_INVALID;
  *info = ctx->last_batch;
  return GMQ_OK;
}

gmq_status gmq_integrate_batch(gmq_context* ctx, int32_t count, const gmq_problem* probs,
                               const double* rel_tols, const gmq_options* opt,
                               int64_t pool_regions, gmq_result* results) {
  NvtxRange range("gmq_integrate_batch");
  if (!ctx || !opt || !results || !probs || count < 1 || count > (1 << 20) ||
      pool_regions < 0 || pool_regions > ((int64_t)1 << 31))
    return GMQ_ERR_INVALID;
  const int64_t cap = opt->max_regions;  // per problem
  if (!(opt->abs_tol >= 0.0) || cap < 1 || cap > kMaxRegions || opt->init_splits < 0 ||
      opt->max_iters < 0 || opt->max_iters > (1 << 28) ||  // the loop bound 4 x max_iters is an int
      (opt->flags & ~GMQ_BATCH_HOST_LOOP) ||
      (opt->precision != GMQ_FP64 && opt->precision != GMQ_MIXED) ||
      (opt->lanes != 0 && opt->lanes != 1 && opt->lanes != 4 && opt->lanes != 32 &&
       opt->lanes != 128) ||
      (opt->precision == GMQ_MIXED && opt->lanes > 1) || opt->rule != GMQ_RULE_GENZ_MALIK ||
      (opt->classifier != GMQ_VOLUME_SHARE && opt->classifier != GMQ_LOCAL_REL) ||
      (opt->estimator != GMQ_EST_EMBEDDED && opt->estimator != GMQ_EST_NULL_RULES))
    return GMQ_ERR_INVALID;
  std::memset(results, 0, sizeof(gmq_result) * (size_t)count);
  const int max_iters = opt->max_iters > 0 ? opt->max_iters : 1000;
  // per-problem descriptors and the initial segments
  std::vector<BatchItem> items((size_t)count);
  bool fam_present[7] = {};
  const bool mixed = opt->precision == GMQ_MIXED;
  int dmax = 1;
  int64_t total = 0;
  // the batch runs in (family, dimension) order, so each family's regions
  // form one contiguous range of every list (the mixed form launches its
  // rule kernel per family over that range); results return in the
  // caller's order, and the order changes no result
  for (int32_t i = 0; i < count; ++i)
    if (validate_problem(&probs[i]) != GMQ_OK) return GMQ_ERR_INVALID;
  std::vector<int32_t> perm((size_t)count);
  for (int32_t i = 0; i < count; ++i) perm[(size_t)i] = i;
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) {
    if (probs[x].family != probs[y].family) return probs[x].family < probs[y].family;
    return probs[x].dim < probs[y].dim;
  });
  int fam_item_lo[8];
  for (int f = 0; f <= 7; ++f) fam_item_lo[f] = count;
  for (int32_t k = count - 1; k >= 0; --k)
    for (int f = 0; f <= probs[perm[(size_t)k]].family; ++f) fam_item_lo[f] = k;
  for (int32_t k = 0; k < count; ++k) {
    const int32_t i = perm[(size_t)k];
    const gmq_problem* p = &probs[i];
    const double tol = rel_tols ? rel_tols[i] : opt->rel_tol;
    if (!(tol >= 0.0)) return GMQ_ERR_INVALID;
    const int d = p->dim;
    dmax = std::max(dmax, d);
    BatchItem& it = items[(size_t)k];
    std::memset(&it, 0, sizeof(it));
    it.P = fam_params(p);
    for (int k = 0; k < GMQ_MAX_DIM; ++k) {
      it.Pf.a[k] = (float)it.P.a[k];
      it.Pf.u[k] = (float)it.P.u[k];
      it.Pf.b[k] = (float)it.P.b[k];
    }
    it.Pf.c0 = (float)it.P.c0;
    fam_present[p->family] = true;
    const RuleConst R = rule_const(d, p->lo, p->hi, opt->estimator);
    for (int c = 0; c < 5; ++c) {
      it.w7[c] = R.w7[c];
      it.w5[c] = R.w5[c];
    }
    for (int c = 0; c < 20; ++c) {
      it.nw[c] = R.nw[c];
    }
    it.vol_omega = R.vol_omega;
    it.rel_tol = tol;
    it.abs_tol = opt->abs_tol;
    it.s = opt->init_splits > 0 ? opt->init_splits : auto_splits(d, cap);
    it.nodes = (int32_t)R.nodes;
    it.cap = cap;
    int64_t n = 1;
    for (int k = 0; k < d; ++k) {
      const double lo = p->lo ? p->lo[k] : 0.0, hi = p->hi ? p->hi[k] : 1.0;
      it.lo[k] = lo;
      it.h0[k] = (hi - lo) / (2.0 * (double)it.s);
      n *= it.s;
      if (n > cap) return GMQ_ERR_INVALID;
    }
    it.off = total;
    it.n = n;
    it.n0 = n;
    total += n;
  }
  // shared pool: the caller's size, or by default the per-problem cap
  // (at least four times the initial partitions)
  const int64_t pool = pool_regions > 0 ? pool_regions : std::max<int64_t>(cap, 4 * total);
  // admission: problems start in index order while their initial
  // partitions fill at most half the pool; the rest wait (deferred, holding
  // no regions) and start when the loop finds room
  total = 0;
  for (int32_t i = 0; i < count; ++i) {
    BatchItem& it = items[(size_t)i];
    // a waiting problem must be able to start in an empty pool
    if (it.n0 > pool / 2) return GMQ_ERR_INVALID;
    if (i == 0 || total + it.n0 <= pool / 2) {
      it.off = total;
      it.n = it.n0;
      total += it.n0;
    } else {
      it.off = 0;
      it.n = 0;
      it.deferred = 1;
    }
  }

  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  // pool: two lists of dmax rows with owner ids, rule outputs, flags,
  // descriptors, loop state
  const int64_t ld = (pool + 31) / 32 * 32;
  const size_t list = align256(sizeof(double) * (size_t)dmax * (size_t)ld);
  const size_t vec = align256(sizeof(double) * (size_t)ld);
  const size_t ids = align256(sizeof(int32_t) * (size_t)ld);
  const size_t bytes = align256((size_t)ld);
  size_t p = 0;
  const size_t o_c0 = p; p += list;
  const size_t o_h0 = p; p += list;
  const size_t o_c1 = p; p += list;
  const size_t o_h1 = p; p += list;
  const size_t o_r0 = p; p += ids;
  const size_t o_r1 = p; p += ids;
  const size_t o_i7 = p; p += 2 * vec;
  const size_t o_err = p; p += 2 * vec;
  const size_t o_vf = p; p += 2 * vec;
  const size_t o_ax = p; p += 2 * bytes;
  const size_t o_fl = p; p += bytes;
  const size_t o_it = p; p += align256(sizeof(BatchItem) * (size_t)count);
  const size_t o_bs = p; p += align256(sizeof(BatchState));
  // tiles: at most pool / kSegTile full tiles plus one short tile per integral
  const int64_t tile_cap = pool / kSegTile + count + 1;
  const size_t toffs = align256(sizeof(long long) * ((size_t)count + 1));
  const size_t tvec = align256(sizeof(double) * (size_t)tile_cap);
  const size_t o_to0 = p; p += toffs;
  const size_t o_to1 = p; p += toffs;
  const size_t o_ta = p; p += tvec;
  const size_t o_tb = p; p += tvec;
  const size_t o_tc = p; p += tvec;
  const size_t o_tp = p; p += tvec;
  char* base = nullptr;
  gmq_status ps = ensure_pool(ctx, p, &base);
  if (ps != GMQ_OK) return ps;
  ctx->part_count = -1;  // the pool no longer holds a kept partition

  BatchArgs B;
  std::memset(&B, 0, sizeof(B));
  B.items = (BatchItem*)(base + o_it);
  B.count = count;
  B.bs = (BatchState*)(base + o_bs);
  B.c[0] = (double*)(base + o_c0);
  B.h[0] = (double*)(base + o_h0);
  B.c[1] = (double*)(base + o_c1);
  B.h[1] = (double*)(base + o_h1);
  B.rid[0] = (int32_t*)(base + o_r0);
  B.rid[1] = (int32_t*)(base + o_r1);
  B.ld = ld;
  B.pool_cap = pool;
  for (int q = 0; q < 2; ++q) {
    B.i7[q] = (double*)(base + o_i7 + q * vec);
    B.err[q] = (double*)(base + o_err + q * vec);
    B.vf[q] = (double*)(base + o_vf + q * vec);
    B.axis[q] = (uint8_t*)(base + o_ax + q * bytes);
  }
  B.flags = (uint8_t*)(base + o_fl);
  B.dmax = dmax;
  B.tile_off[0] = (long long*)(base + o_to0);
  B.tile_off[1] = (long long*)(base + o_to1);
  B.tile_a = (double*)(base + o_ta);
  B.tile_b = (double*)(base + o_tb);
  B.tile_cnt = (long long*)(base + o_tc);
  B.tile_pos = (long long*)(base + o_tp);
  B.tile_grid = 2 * ctx->sm_count;
  B.classifier = opt->classifier;
  B.estimator = opt->estimator;
  B.guard = mixed ? kGuardMixed : kGuardFp64;
  const RuleConst R0 = rule_const(1, nullptr, nullptr);
  B.lam2 = R0.lam2;
  B.lam3 = R0.lam3;
  B.lam5 = R0.lam5;
  B.ratio = R0.ratio;
  BatchState bs0;
  std::memset(&bs0, 0, sizeof(bs0));
  bs0.n_total = total;
  bs0.active = count;
  bs0.max_iters = max_iters;
  // pauses (pool full) add sweeps; the device loop is bounded all the same
  bs0.max_sweeps = 4 * max_iters;
  cudaStream_t strm = ctx->stream;
  // the initial list's tile table
  std::vector<long long> toff0((size_t)count + 1);
  long long ntiles = 0;
  for (int32_t i = 0; i < count; ++i) {
    toff0[(size_t)i] = ntiles;
    ntiles += (items[(size_t)i].n + kSegTile - 1) / kSegTile;
  }
  toff0[(size_t)count] = ntiles;
  bs0.n_tiles = ntiles;
  // first region of each family in the initial list
  {
    long long pos = 0;
    int f = 0;
    for (int32_t k = 0; k <= count; ++k) {
      while (f < 8 && fam_item_lo[f] == k) bs0.fam_off[0][f++] = pos;
      if (k < count) pos += items[(size_t)k].n;
    }
    while (f < 8) bs0.fam_off[0][f++] = pos;
  }
  for (int f = 0; f < 8; ++f) B.fam_item_lo[f] = fam_item_lo[f];
  GMQ_CK(cudaMemcpyAsync(B.tile_off[0], toff0.data(), sizeof(long long) * ((size_t)count + 1),
                         cudaMemcpyHostToDevice, strm));
  GMQ_CK(cudaMemcpyAsync(B.items, items.data(), sizeof(BatchItem) * (size_t)count,
                         cudaMemcpyHostToDevice, strm));
  GMQ_CK(cudaMemcpyAsync(B.bs, &bs0, sizeof(BatchState), cudaMemcpyHostToDevice, strm));
  GMQ_CK(batch_launch_partition(B, strm));
  ctx->launches += 1;

  // lanes per region of the rule kernel: forced, or per sweep from the list
  // length with thresholds the autotuner sets once per largest dimension by
  // timing the three mappings on copies of the initial list (the launches
  // only write rule outputs, which the first sweep overwrites)
  gmq_batch_info info;
  std::memset(&info, 0, sizeof(info));
  // one rule launch per family present (FP64: lanes per region per sweep;
  // mixed: one lane per region), each a persistent grid of its own size
  int fam_grid[7] = {};
  for (int f = 0; f < 7; ++f)
    if (fam_present[f])
      fam_grid[f] = ctx->sm_count * (mixed ? batch_rule_mixed_max_blocks(f, dmax)
                                           : batch_rule64_max_blocks(f, dmax));
  auto launch_rule_step = [&](cudaStream_t st) -> cudaError_t {
    for (int f = 0; f < 7; ++f) {
      if (!fam_present[f]) continue;
      const cudaError_t e = mixed ? batch_launch_rule_mixed(f, B, fam_grid[f], st)
                                  : batch_launch_rule64(f, B, fam_grid[f], st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  int rule_launches = 0;
  for (int f = 0; f < 7; ++f) rule_launches += fam_present[f] ? 1 : 0;
  // the family the autotuner times (its kernel over copies of the whole
  // initial list stands for the rule step: the lanes choice depends on the
  // list length and the dimension, not on the integrand)
  int f_tune = 0;
  while (f_tune < 6 && !fam_present[f_tune]) ++f_tune;
  const int grid = fam_grid[f_tune];
  B.forced_lanes = mixed ? 1 : opt->lanes;
  if (!mixed && !opt->lanes && !ctx->tuned[dmax]) {
    const int64_t wave = (int64_t)grid * kBatchRuleBlock;  // regions of one T = 1 wave
    int64_t lens[5];
    int nl = 0;
    for (int64_t L : {wave / 64, wave / 16, wave / 4, wave, 4 * wave}) {
      L = std::min<int64_t>(std::max<int64_t>(L, 1), pool);
      if (nl == 0 || L > lens[nl - 1]) lens[nl++] = L;
    }
    GMQ_CK(batch_launch_tile(B, total, lens[nl - 1], strm));
    ctx->launches += 1;
    const int modes[4] = {1, 4, 32, 128};
    int best[5];
    EventPair ev;  // destroyed on every return path
    GMQ_CK(cudaEventCreate(&ev.a));
    GMQ_CK(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    for (int i = 0; i < nl; ++i) {
      float mbest = 1e30f;
      float ms[4];
      for (int m = 0; m < 4; ++m) {
        BatchState t = bs0;
        t.n_total = lens[i];
        t.lanes = modes[m];
        for (int f = 0; f < 8; ++f) t.fam_off[0][f] = f <= f_tune ? 0 : lens[i];
        GMQ_CK(cudaMemcpyAsync(B.bs, &t, sizeof(BatchState), cudaMemcpyHostToDevice, strm));
        GMQ_CK(batch_launch_rule64(f_tune, B, grid, strm));  // warm-up
        GMQ_CK(cudaEventRecord(e0, strm));
        GMQ_CK(batch_launch_rule64(f_tune, B, grid, strm));
        GMQ_CK(cudaEventRecord(e1, strm));
        GMQ_CK(cudaEventSynchronize(e1));
        GMQ_CK(cudaEventElapsedTime(&ms[m], e0, e1));
        ctx->launches += 2;
        info.tune_ms[i][m] = ms[m];
        mbest = std::min(mbest, ms[m]);
      }
      // the fewest lanes within 5% of the fastest mapping
      best[i] = 3;
      for (int m = 3; m >= 0; --m)
        if (ms[m] <= 1.05f * mbest) best[i] = m;
      info.tune_n[i] = lens[i];
    }
    auto between = [&](int i) -> long long {  // geometric middle of lens[i-1], lens[i]
      return (long long)std::llround(std::sqrt((double)lens[i - 1] * (double)lens[i]));
    };
    // one lane from the shortest timed length where it wins there and at
    // every longer one (beyond twice the longest if it never does)
    int i1 = nl;
    for (int i = nl - 1; i >= 0 && best[i] == 0; --i) i1 = i;
    const long long t1 = i1 == nl ? 2 * lens[nl - 1] : (i1 == 0 ? 0 : between(i1));
    int i4 = i1;
    for (int i = i1 - 1; i >= 0 && best[i] <= 1; --i) i4 = i;
    const long long t4 = i4 == i1 ? t1 : (i4 == 0 ? 0 : between(i4));
    int i32 = i4;
    for (int i = i4 - 1; i >= 0 && best[i] <= 2; --i) i32 = i;
    const long long t32 = i32 == i4 ? t4 : (i32 == 0 ? 0 : between(i32));
    ctx->tuned[dmax] = 1;
    ctx->tuned_t1[dmax] = t1;
    ctx->tuned_t4[dmax] = t4;
    ctx->tuned_t32[dmax] = t32;
    info.autotuned = 1;
  }
  B.lanes_t1 = ctx->tuned_t1[dmax];
  B.lanes_t4 = ctx->tuned_t4[dmax];
  B.lanes_t32 = ctx->tuned_t32[dmax];
  bs0.lanes = batch_lanes_for(B, bs0.n_total);
  GMQ_CK(cudaMemcpyAsync(B.bs, &bs0, sizeof(BatchState), cudaMemcpyHostToDevice, strm));
  info.rule_block = kBatchRuleBlock;
  info.rule_grid = 0;
  for (int f = 0; f < 7; ++f) info.rule_grid = std::max(info.rule_grid, fam_grid[f]);
  info.forced_lanes = B.forced_lanes;
  info.lanes_t1 = B.forced_lanes ? 0 : B.lanes_t1;
  info.lanes_t4 = B.forced_lanes ? 0 : B.lanes_t4;
  info.lanes_t32 = B.forced_lanes ? 0 : B.lanes_t32;

  BatchState hs;
  if (!(opt->flags & GMQ_BATCH_HOST_LOOP)) {
    // one graph: a while node whose body is one sweep; the last kernel of
    // the body sets the condition (false once every problem has stopped or
    // max_iters sweeps ran)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    cudaGraphConditionalHandle handle = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&handle, graph, 1,
                                                                cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, graph, nullptr, nullptr, 0, &cp);
    if (e == cudaSuccess) {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      B.cond = handle;
      B.use_cond = 1;
      // capture on the context's private stream: the caller's stream may be
      // the legacy default stream, which cannot be captured; capturing runs
      // nothing, the graph is launched on the caller's stream below
      if (!ctx->capture_stream)
        e = cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(ctx->capture_stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t e1 = launch_rule_step(ctx->capture_stream);
        cudaError_t e2 = batch_launch_rest(B, ctx->capture_stream);
        cudaGraph_t captured = nullptr;
        e = cudaStreamEndCapture(ctx->capture_stream, &captured);
        if (e == cudaSuccess) e = (e1 != cudaSuccess) ? e1 : e2;
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, strm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e);
    ctx->launches += 1;
    info.used_graph = 1;
  } else {
    B.use_cond = 0;
    for (;;) {
      for (int k = 0; k < 8; ++k) {
        GMQ_CK(launch_rule_step(strm));
        GMQ_CK(batch_launch_rest(B, strm));
        ctx->launches += 7 + rule_launches;
      }
      GMQ_CK(cudaMemcpyAsync(ctx->h_status, B.bs, sizeof(BatchState), cudaMemcpyDeviceToHost,
                             strm));
      GMQ_CK(cudaStreamSynchronize(strm));
      std::memcpy(&hs, ctx->h_status, sizeof(BatchState));
      if (hs.active == 0 || hs.sweep >= hs.max_sweeps) break;
    }
  }
  GMQ_CK(cudaMemcpyAsync(ctx->h_status, B.bs, sizeof(BatchState), cudaMemcpyDeviceToHost, strm));
  GMQ_CK(cudaMemcpyAsync(items.data(), B.items, sizeof(BatchItem) * (size_t)count,
                         cudaMemcpyDeviceToHost, strm));
  GMQ_CK(cudaStreamSynchronize(strm));
  std::memcpy(&hs, ctx->h_status, sizeof(BatchState));
  info.sweeps = hs.sweep;
  info.pauses = hs.pauses;
  info.evictions = hs.evictions;
  info.rule_regions = hs.rule_regions;
  info.carried_regions = hs.carried_regions;
  info.list_regions = hs.list_regions;
  for (int m = 0; m < 4; ++m) info.lane_sweeps[m] = hs.lane_sweeps[m];
  ctx->last_batch = info;
  for (int32_t k = 0; k < count; ++k) {
    const BatchItem& it = items[(size_t)k];
    gmq_result& r = results[perm[(size_t)k]];
    r.integral = it.I;
    r.error = it.E;
    r.regions_evaluated = it.regions;
    r.function_evals = it.regions * (int64_t)it.nodes;
    r.final_active = it.n;
    r.iterations = it.iters;
    if (it.flags & kNonfinite)
      r.status = GMQ_ERR_NONFINITE;
    else if (it.flags & kConverged)
      r.status = GMQ_OK;
    else if (it.flags & kLastSweep)
      r.status = GMQ_MAX_ITERS;
    else if (it.flags & kAllRetired)
      r.status = GMQ_ROUNDOFF_LIMIT;
    else if (it.flags & kCapExceeded)
      r.status = GMQ_CAP_REACHED;
    else
      r.status = GMQ_MAX_ITERS;
  }
  return GMQ_OK;
}

gmq_status gmq_rule_grad(gmq_context* ctx, const gmq_problem* prob, int64_t n,
                         const double* d_center, const double* d_halfw, int64_t ld,
                         double* integral, double* grad) {
  NvtxRange range("gmq_rule_grad");
  if (!ctx || !integral || !grad) return GMQ_ERR_INVALID;
  gmq_status vs = validate_problem(prob);
  if (vs != GMQ_OK) return vs;
  const int d = prob->dim;
  if (n < 0 || n > kMaxRegions || ld < n || (n > 0 && (!d_center || !d_halfw)))
    return GMQ_ERR_INVALID;
  *integral = 0.0;
  for (int k = 0; k < 2 * d; ++k) grad[k] = 0.0;
  if (n == 0) return GMQ_OK;
  DeviceGuard g(ctx->device);
  if (!g.ok) return GMQ_ERR_CUDA;
  // working memory: per-region contributions [2d+1][ldo], per-row tile
  // partials, row tickets and row sums
  const int rows = 2 * d + 1;
  const int64_t ldo = (n + 31) / 32 * 32;
  const int64_t nb = (n + kTile - 1) / kTile;
  const size_t o_out = 0;
  const size_t o_blk = o_out + align256(sizeof(double) * (size_t)rows * (size_t)ldo);
  const size_t o_tk = o_blk + align256(sizeof(double) * (size_t)rows * (size_t)nb);
  const size_t o_sum = o_tk + align256(sizeof(unsigned) * (size_t)rows);
  const size_t need = o_sum + align256(sizeof(double) * (size_t)rows);
  if (ctx->gscratch_bytes < need) {
    if (ctx->gscratch) cudaFree(ctx->gscratch);
    ctx->gscratch = nullptr;
    ctx->gscratch_bytes = 0;
    void* q = nullptr;
    if (cudaMalloc(&q, need) != cudaSuccess) {
      cudaGetLastError();
      return GMQ_ERR_OOM;
    }
    ctx->gscratch = (char*)q;
    ctx->gscratch_bytes = need;
  }
  char* b = ctx->gscratch;
  GradArgs A;
  A.c = d_center;
  A.h = d_halfw;
  A.ld = ld;
  A.n = n;
  A.out = (double*)(b + o_out);
  A.ldo = ldo;
  A.P = fam_params(prob);
  A.R = rule_const(d, prob->lo, prob->hi);
  A.nodewise = ctx->eval_mode == GMQ_EVAL_NODEWISE ? 1 : 0;
  cudaStream_t strm = ctx->stream;
  cudaError_t e;
  prof_begin(ctx, kKRule);
  switch (prob->family) {
    case GMQ_OSCILLATORY: e = launch_rule_grad_family<GMQ_OSCILLATORY>(A, strm); break;
    case GMQ_PRODUCT_PEAK: e = launch_rule_grad_family<GMQ_PRODUCT_PEAK>(A, strm); break;
    case GMQ_CORNER_PEAK: e = launch_rule_grad_family<GMQ_CORNER_PEAK>(A, strm); break;
    case GMQ_GAUSSIAN: e = launch_rule_grad_family<GMQ_GAUSSIAN>(A, strm); break;
    case GMQ_C0: e = launch_rule_grad_family<GMQ_C0>(A, strm); break;
    case GMQ_DISCONTINUOUS: e = launch_rule_grad_family<GMQ_DISCONTINUOUS>(A, strm); break;
    default: e = launch_rule_grad_family<GMQ_POLY_SUMSQ11>(A, strm); break;
  }
  GMQ_CK(e);
  prof_end(ctx, kKRule, n);
  GMQ_CK(cudaMemsetAsync(b + o_tk, 0, sizeof(unsigned) * (size_t)rows, strm));
  prof_begin(ctx, kKSum);
  GMQ_CK(launch_rows_tree_sum(A.out, ldo, n, rows, (double*)(b + o_blk), (unsigned*)(b + o_tk),
                              (double*)(b + o_sum), strm));
  prof_end(ctx, kKSum, n);
  ctx->launches += 2;
  std::vector<double> sums((size_t)rows);
  GMQ_CK(cudaMemcpyAsync(sums.data(), b + o_sum, sizeof(double) * (size_t)rows,
                         cudaMemcpyDeviceToHost, strm));
  GMQ_CK(cudaStreamSynchronize(strm));
  prof_collect(ctx);
  for (int k = 0; k < 2 * d; ++k) grad[k] = sums[(size_t)k];
  *integral = sums[(size_t)(2 * d)];
  return GMQ_OK;
}

}  // extern "C"
