// gm_adjoint.cuh -- adjoint of the rule over a frozen partition.
//
// For a fixed set of regions (the leaves an adaptive integration ended
// with), the quadrature value is Q(theta) = sum_r vol_r sum_i w_i f(x_i;
// theta), with the degree-7 Genz-Malik weights w_i of the node's class.
// Its exact gradient with respect to the integrand parameters theta =
// (a_1..a_d, u_1..u_d) is the same rule applied to df/dtheta:
//   dQ/dtheta_k = sum_r vol_r sum_i w_i df/dtheta_k(x_i).
// k_rule_grad_sep (the default) forms the gradient from per-axis, per-row
// sums of w_i g'(S_i) over the separable form; k_rule_grad
// (GMQ_EVAL_NODEWISE) evaluates f and its 2d parameter derivatives at every
// node from a node-coordinate table.  Both run a thread per region, write
// the region's contributions (and its I7) to a [2d+1][n] array, and the
// per-row pairwise-tree sums give Q and its gradient.
#pragma once

#include "gm_rule.cuh"

namespace gmq {

struct GradArgs {
  const double* c;
  const double* h;
  int64_t ld;
  int64_t n;
  double* out;     // [2d+1][ldo]: rows 0..d-1 dQ/da, d..2d-1 dQ/du, 2d I7
  int64_t ldo;
  FamParams P;
  RuleConst R;
  int32_t nodewise;  // 1: k_rule_grad (f and its derivatives node by node)
};

// f and w * df/dtheta accumulated into ga[j] (a_j) and gu[j] (u_j); the
// accumulators are per-thread shared-memory rows with stride `st`.
template <int FAM>
struct FamilyGrad;

template <>
struct FamilyGrad<GMQ_OSCILLATORY> {
  template <class X>
  __device__ static double eval(const SmemParams<double>& P, int d, X x, double w, double* ga,
                                double* gu, int st) {
    double s = P.c0;
    for (int j = 0; j < d; ++j) s = fma(P.a[j], x(j), s);
    double sn, cs;
    sincos(s, &sn, &cs);
    const double ws = -w * sn;
    for (int j = 0; j < d; ++j) ga[j * st] = fma(ws, x(j), ga[j * st]);
    gu[0] = fma(ws, 2.0 * M_PI, gu[0]);  // d s / d u_1 = 2 pi
    return cs;
  }
};

template <>
struct FamilyGrad<GMQ_PRODUCT_PEAK> {
  template <class X>
  __device__ static double eval(const SmemParams<double>& P, int d, X x, double w, double* ga,
                                double* gu, int st) {
    double den = 1.0;
    for (int j = 0; j < d; ++j) {
      const double t = x(j) - P.u[j];
      den *= fma(t, t, P.b[j]);
    }
    const double f = 1.0 / den;
    const double wf = w * f;
    for (int j = 0; j < d; ++j) {
      const double t = x(j) - P.u[j];
      const double q = 1.0 / fma(t, t, P.b[j]);
      // b_j = a_j^-2: df/da_j = 2 f a_j^-3 q, df/du_j = 2 f t q
      const double ainv = 1.0 / P.a[j];
      ga[j * st] = fma(wf, 2.0 * ainv * ainv * ainv * q, ga[j * st]);
      gu[j * st] = fma(wf, 2.0 * t * q, gu[j * st]);
    }
    return f;
  }
};

template <>
struct FamilyGrad<GMQ_CORNER_PEAK> {
  template <class X>
  __device__ static double eval(const SmemParams<double>& P, int d, X x, double w, double* ga,
                                double* gu, int st) {
    double s = 1.0;
    for (int j = 0; j < d; ++j) s = fma(P.a[j], x(j), s);
    const double f = 1.0 / ipow(s, d + 1);
    const double c = -w * (double)(d + 1) * f / s;  // df/da_j = -(d+1) x_j f / s
    for (int j = 0; j < d; ++j) ga[j * st] = fma(c, x(j), ga[j * st]);
    return f;
  }
};

template <>
struct FamilyGrad<GMQ_GAUSSIAN> {
  template <class X>
  __device__ static double eval(const SmemParams<double>& P, int d, X x, double w, double* ga,
                                double* gu, int st) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
      const double t = x(j) - P.u[j];
      s = fma(P.b[j], t * t, s);
    }
    const double f = exp(-s);
    const double wf = w * f;
    for (int j = 0; j < d; ++j) {
      const double t = x(j) - P.u[j];
      // df/da_j = -2 a_j t^2 f, df/du_j = 2 a_j^2 t f
      ga[j * st] = fma(wf, -2.0 * P.a[j] * t * t, ga[j * st]);
      gu[j * st] = fma(wf, 2.0 * P.b[j] * t, gu[j * st]);
    }
    return f;
  }
};

template <>
struct FamilyGrad<GMQ_C0> {
  template <class X>
  __device__ static double eval(const SmemParams<double>& P, int d, X x, double w, double* ga,
                                double* gu, int st) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) s = fma(P.a[j], fabs(x(j) - P.u[j]), s);
    const double f = exp(-s);
    const double wf = w * f;
    for (int j = 0; j < d; ++j) {
      const double t = x(j) - P.u[j];
      const double sg = (t > 0.0) ? 1.0 : ((t < 0.0) ? -1.0 : 0.0);
      // df/da_j = -|t| f, df/du_j = a_j sign(t) f
      ga[j * st] = fma(wf, -fabs(t), ga[j * st]);
      gu[j * st] = fma(wf, P.a[j] * sg, gu[j * st]);
    }
    return f;
  }
};

template <>
struct FamilyGrad<GMQ_DISCONTINUOUS> {
  template <class X>
  __device__ static double eval(const SmemParams<double>& P, int d, X x, double w, double* ga,
                                double* gu, int st) {
    double s = 0.0;
    bool zero = false;
    for (int j = 0; j < d; ++j) {
      const double xj = x(j);
      zero = zero || (xj > P.u[j]);
      s = fma(P.a[j], xj, s);
    }
    if (zero) return 0.0;
    const double f = exp(s);
    const double wf = w * f;
    // df/da_j = x_j f; the thresholds u_j move a discontinuity, whose
    // contribution a frozen partition does not see (df/du_j = 0 a.e.)
    for (int j = 0; j < d; ++j) ga[j * st] = fma(wf, x(j), ga[j * st]);
    return f;
  }
};

template <>
struct FamilyGrad<GMQ_POLY_SUMSQ11> {
  template <class X>
  __device__ static double eval(const SmemParams<double>& P, int d, X x, double, double*, double*,
                                int) {
    return Family<GMQ_POLY_SUMSQ11>::template eval<double>(P, d, x);
  }
};

// Separable adjoint (the default; GMQ_EVAL_NODEWISE keeps k_rule_grad).
// With f = g(S), S = base (+) phi_0(x_0) (+) ... (Sep<FAM>), df/dtheta_j at a
// node is D(S) c_j(x_j): D = g'(S) and c_j = dphi_j/dtheta_j for the additive
// families; for the product peak (f = 1/prod psi_j) D = f and c_j =
// -(dpsi_j/dtheta_j) / psi_j.  A node's coordinate on axis j is one of
// seven values, so
//   dQ/dtheta_j = vol sum_rows c_j(x_row) H[j][row],
//   H[j][row] = sum of w_i D(S_i) over the nodes with x_ij = x_row,
// and a node only adds w D into one or two sums: its class-2/3 slot, the
// two axis slots of a pair node, or (sign-pattern nodes) a per-pattern-low-
// bits and a per-block table from which the per-axis sums follow.  The
// centre rows are the totals minus the other rows.  The oscillatory base
// 2 pi u_1 adds 2 pi sum_i w_i D_i to dQ/du_1.
template <int FAM>
struct SepGrad;

template <>
struct SepGrad<GMQ_OSCILLATORY> {
  __device__ static void fd(int, double S, double& f, double& D) {
    double sn, cs;
    gm_sincos(S, &sn, &cs);
    f = cs;
    D = -sn;
  }
  __device__ static void coef(const SmemParams<double>&, int, double x, double& ca, double& cu) {
    ca = x;
    cu = 0.0;
  }
};

template <>
struct SepGrad<GMQ_PRODUCT_PEAK> {
  __device__ static void fd(int, double S, double& f, double& D) {
    f = gm_rcp(S);
    D = f;
  }
  __device__ static void coef(const SmemParams<double>& P, int j, double x, double& ca,
                              double& cu) {
    // b_j = a_j^-2: dpsi/da_j = -2 a_j^-3, dpsi/du_j = -2 t
    const double t = __dsub_rn(x, P.u[j]);
    const double q = gm_rcp(fma(t, t, P.b[j]));
    const double ainv = gm_rcp(P.a[j]);
    ca = __dmul_rn(__dmul_rn(2.0, __dmul_rn(ainv, __dmul_rn(ainv, ainv))), q);
    cu = __dmul_rn(__dmul_rn(2.0, t), q);
  }
};

template <>
struct SepGrad<GMQ_CORNER_PEAK> {
  __device__ static void fd(int d, double S, double& f, double& D) {
    f = gm_rcp(ipow(S, d + 1));
    D = __dmul_rn(__dmul_rn(-(double)(d + 1), f), gm_rcp(S));
  }
  __device__ static void coef(const SmemParams<double>&, int, double x, double& ca, double& cu) {
    ca = x;
    cu = 0.0;
  }
};

template <>
struct SepGrad<GMQ_GAUSSIAN> {
  __device__ static void fd(int, double S, double& f, double& D) {
    f = gm_exp(-S);
    D = -f;
  }
  __device__ static void coef(const SmemParams<double>& P, int j, double x, double& ca,
                              double& cu) {
    // phi = a^2 t^2: dphi/da = 2 a t^2, dphi/du = -2 a^2 t
    const double t = __dsub_rn(x, P.u[j]);
    ca = __dmul_rn(__dmul_rn(2.0, P.a[j]), __dmul_rn(t, t));
    cu = __dmul_rn(__dmul_rn(-2.0, P.b[j]), t);
  }
};

template <>
struct SepGrad<GMQ_C0> {
  __device__ static void fd(int, double S, double& f, double& D) {
    f = gm_exp(-S);
    D = -f;
  }
  __device__ static void coef(const SmemParams<double>& P, int j, double x, double& ca,
                              double& cu) {
    // phi = a |t|: dphi/da = |t|, dphi/du = -a sign(t)
    const double t = __dsub_rn(x, P.u[j]);
    ca = fabs(t);
    cu = t > 0.0 ? -P.a[j] : (t < 0.0 ? P.a[j] : 0.0);
  }
};

template <>
struct SepGrad<GMQ_DISCONTINUOUS> {
  __device__ static void fd(int, double S, double& f, double& D) {
    f = gm_exp(S);
    D = f;
  }
  __device__ static void coef(const SmemParams<double>&, int, double x, double& ca, double& cu) {
    ca = x;
    cu = 0.0;  // the thresholds move a jump, which a frozen partition does not see
  }
};

template <>
struct SepGrad<GMQ_POLY_SUMSQ11> {
  __device__ static void fd(int d, double S, double& f, double& D) {
    f = Sep<GMQ_POLY_SUMSQ11>::g(d, S);
    D = 0.0;  // no parameters
  }
  __device__ static void coef(const SmemParams<double>&, int, double, double& ca, double& cu) {
    ca = 0.0;
    cu = 0.0;
  }
};

constexpr int kGradSepBlock = 64;

// Per-thread shared-memory words of the separable adjoint: the rule's
// separable workspace, then the class-2/3 node terms [4d], the pair-node
// sums per axis and sign [2d] and the sign-pattern tables [2^a + 2^b + 2^c].
__host__ __device__ inline int grad_sep_words(int d, bool flag) {
  const int a = sep_a(d), b = sep_b(d), c = sep_c(d);
  return sep_layout(d, flag, false).words + 4 * d + 2 * d + (1 << a) + (b ? 1 << b : 0) +
         (c ? 1 << c : 0);
}

inline size_t grad_sep_smem_bytes(int d, bool flag) {
  return sizeof(double) * (size_t)grad_sep_words(d, flag) * kGradSepBlock +
         sizeof(SmemParams<double>) + 16;
}

template <int FAM>
__global__ void __launch_bounds__(kGradSepBlock) k_rule_grad_sep(const GradArgs A) {
  using SF = Sep<FAM>;
  using SG = SepGrad<FAM>;
  constexpr int RB = kGradSepBlock;
  extern __shared__ __align__(16) double smem[];
  const int d = A.P.d;
  const SepLayout Ly = sep_layout(d, SF::kFlag, false);
  const int words = grad_sep_words(d, SF::kFlag);
  SmemParams<double>* P = reinterpret_cast<SmemParams<double>*>(smem + (size_t)words * RB);
  const int tid = threadIdx.x;
  for (int j = tid; j < d; j += RB) {
    P->a[j] = A.P.a[j];
    P->u[j] = A.P.u[j];
    P->b[j] = A.P.b[j];
  }
  if (tid == 0) P->c0 = A.P.c0;
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * RB + tid;
  if (r >= A.n) return;
  double* w = smem + tid;
  auto W = [&](int e) -> double& { return w[(long long)e * RB]; };
  const int eHA = Ly.words, eG4 = eHA + 4 * d, eTL = eG4 + 2 * d;
  const int pa = sep_a(d), pb = sep_b(d), pc = sep_c(d);
  const int eTB = eTL + (1 << pa), eTC = eTB + (pb ? 1 << pb : 0);
  const double* C = A.c + r;
  const double* H = A.h + r;
  const int64_t ld = A.ld;
  auto ch = [&](int k, double& c, double& h) {
    c = C[(int64_t)k * ld];
    h = H[(int64_t)k * ld];
  };
  auto op = [](double x, double y) -> double {
    if constexpr (SF::kMul)
      return __dmul_rn(x, y);
    else
      return __dadd_rn(x, y);
  };
  // f and D at S; a node that the discontinuous family zeroes gives 0, 0
  auto node = [&](double S, bool zero, double& f, double& D) {
    if constexpr (SF::kFlag) {
      if (zero) {
        f = 0.0;
        D = 0.0;
        return;
      }
    }
    SG::fd(d, S, f, D);
  };
  const double lam2 = A.R.lam2, lam3 = A.R.lam3, lam5 = A.R.lam5;
  const double* w7 = A.R.w7;
  unsigned zc = 0u, z3 = 0u, z5 = 0u;
  // right to left: phi at the centre, R, suf (suf_{k+1} parked in L[k][0])
  double suf = 0.0;
  for (int k = d - 1; k >= 0; --k) {
    double c, h;
    ch(k, c, h);
    const double xp = fma(lam3, h, c), xm = fma(-lam3, h, c);
    const double fc = SF::phi(*P, k, c), fp = SF::phi(*P, k, xp), fm = SF::phi(*P, k, xm);
    if constexpr (SF::kFlag) {
      zc |= (unsigned)SF::flag(*P, k, c) << k;
      z3 |= ((unsigned)SF::flag(*P, k, xp) << k) | ((unsigned)SF::flag(*P, k, xm) << (k + 16));
    }
    W(Ly.phiC + k) = fc;
    if (k == d - 1) {
      W(Ly.R + 2 * k) = fp;
      W(Ly.R + 2 * k + 1) = fm;
      suf = fc;
    } else {
      W(Ly.R + 2 * k) = op(fp, suf);
      W(Ly.R + 2 * k + 1) = op(fm, suf);
      W(Ly.L + 2 * k) = suf;
      suf = op(fc, suf);
    }
  }
  double s1, s2 = 0.0, s3 = 0.0, s4 = 0.0, s5 = 0.0;  // class sums of f
  double hC, T23 = 0.0, T4 = 0.0, T5 = 0.0;          // sums of w D
  {
    double f, D;
    node(SF::kBase ? op(SF::base(*P), suf) : suf, zc != 0u, f, D);
    s1 = f;
    hC = __dmul_rn(w7[0], D);
  }
  // left to right: the axis nodes and the pair-node prefixes L
  double pre = SF::kBase ? SF::base(*P) : 0.0;
  bool hp = SF::kBase;
  for (int k = 0; k < d; ++k) {
    double c, h;
    ch(k, c, h);
    const bool hs = k < d - 1;
    const double sk = hs ? W(Ly.L + 2 * k) : 0.0;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const double lam = rr < 2 ? (rr ? -lam2 : lam2) : (rr == 2 ? lam3 : -lam3);
      const double x = fma(lam, h, c);
      const double ph = SF::phi(*P, k, x);
      const double lp = hp ? op(pre, ph) : ph;
      if (rr >= 2) W(Ly.L + 2 * k + (rr - 2)) = lp;
      bool zero = false;
      if constexpr (SF::kFlag) zero = ((zc & ~(1u << k)) != 0u) || SF::flag(*P, k, x);
      double f, D;
      node(hs ? op(lp, sk) : lp, zero, f, D);
      const double hw = __dmul_rn(w7[rr < 2 ? 1 : 2], D);
      if (rr < 2)
        s2 = __dadd_rn(s2, f);
      else
        s3 = __dadd_rn(s3, f);
      W(eHA + 4 * k + rr) = hw;
      T23 = __dadd_rn(T23, hw);
    }
    const double fck = W(Ly.phiC + k);
    pre = hp ? op(pre, fck) : fck;
    hp = true;
    W(eG4 + 2 * k) = 0.0;
    W(eG4 + 2 * k + 1) = 0.0;
  }
  // class-5 chains by doubling (as the rule kernel forms them)
  auto chains = [&](int e0, int j0, int nb, bool with_base) {
    for (int i = 0; i < nb; ++i) {
      double c, h;
      ch(j0 + i, c, h);
      const double xp = fma(lam5, h, c), xm = fma(-lam5, h, c);
      const double fp = SF::phi(*P, j0 + i, xp), fm = SF::phi(*P, j0 + i, xm);
      if constexpr (SF::kFlag)
        z5 |= ((unsigned)SF::flag(*P, j0 + i, xp) << (j0 + i)) |
              ((unsigned)SF::flag(*P, j0 + i, xm) << (j0 + i + 16));
      if (i == 0) {
        W(e0) = with_base ? op(SF::base(*P), fp) : fp;
        W(e0 + 1) = with_base ? op(SF::base(*P), fm) : fm;
      } else {
        const int n = 1 << i;
        for (int t = 0; t < n; ++t) {
          const double v = W(e0 + t);
          W(e0 + t + n) = op(v, fm);
          W(e0 + t) = op(v, fp);
        }
      }
    }
  };
  chains(Ly.A, 0, pa, SF::kBase);
  if (pb) chains(Ly.B, pa, pb, false);
  if (pc) chains(Ly.C, pa + pb, pc, false);
  // class 4: pairs j < k in lexicographic order, signs ++, +-, -+, --
  for (int j = 0; j < d - 1; ++j) {
    double mid = 0.0;
    bool hmid = false;
    for (int k = j + 1; k < d; ++k) {
      if (k > j + 1) {
        const double t = W(Ly.phiC + k - 1);
        mid = hmid ? op(mid, t) : t;
        hmid = true;
      }
      double gk0 = 0.0, gk1 = 0.0;
#pragma unroll
      for (int sj = 0; sj < 2; ++sj) {
        const double L = W(Ly.L + 2 * j + sj);
        const double lm = hmid ? op(L, mid) : L;
        double gj = 0.0;
#pragma unroll
        for (int sk = 0; sk < 2; ++sk) {
          bool zero = false;
          if constexpr (SF::kFlag)
            zero = ((zc & ~((1u << j) | (1u << k))) != 0u) || ((z3 >> (j + 16 * sj)) & 1u) ||
                   ((z3 >> (k + 16 * sk)) & 1u);
          double f, D;
          node(op(lm, W(Ly.R + 2 * k + sk)), zero, f, D);
          s4 = __dadd_rn(s4, f);
          const double hw = __dmul_rn(w7[3], D);
          gj = __dadd_rn(gj, hw);
          if (sk)
            gk1 = __dadd_rn(gk1, hw);
          else
            gk0 = __dadd_rn(gk0, hw);
        }
        W(eG4 + 2 * j + sj) = __dadd_rn(W(eG4 + 2 * j + sj), gj);
        T4 = __dadd_rn(T4, gj);
      }
      W(eG4 + 2 * k) = __dadd_rn(W(eG4 + 2 * k), gk0);
      W(eG4 + 2 * k + 1) = __dadd_rn(W(eG4 + 2 * k + 1), gk1);
    }
  }
  // class 5: sign patterns m = lo + 2^a q (bit j set: -lambda5 on axis j);
  // w D goes to TL[lo] and, summed over the block, to TB[q's low b bits]
  // and TC[q's high bits]
  const int nlo = 1 << pa, nq = 1 << (d - pa);
  for (int t = 0; t < nlo; ++t) W(eTL + t) = 0.0;
  for (int t = 0; t < (pb ? 1 << pb : 0); ++t) W(eTB + t) = 0.0;
  for (int t = 0; t < (pc ? 1 << pc : 0); ++t) W(eTC + t) = 0.0;
  const unsigned dmask = (1u << d) - 1u;
  for (int q = 0; q < nq; ++q) {
    double bc = 0.0;
    if (pb) bc = pc ? op(W(Ly.B + (q & ((1 << pb) - 1))), W(Ly.C + (q >> pb))) : W(Ly.B + q);
    double U = 0.0;
    for (int lo = 0; lo < nlo; ++lo) {
      const double S = pb ? op(W(Ly.A + lo), bc) : W(Ly.A + lo);
      bool zero = false;
      if constexpr (SF::kFlag) {
        const unsigned m = (unsigned)lo | ((unsigned)q << pa);
        zero = ((((~m) & z5) | (m & (z5 >> 16))) & dmask) != 0u;
      }
      double f, D;
      node(S, zero, f, D);
      s5 = __dadd_rn(s5, f);
      const double hw = __dmul_rn(w7[4], D);
      W(eTL + lo) = __dadd_rn(W(eTL + lo), hw);
      U = __dadd_rn(U, hw);
    }
    if (pb) W(eTB + (q & ((1 << pb) - 1))) = __dadd_rn(W(eTB + (q & ((1 << pb) - 1))), U);
    if (pc) W(eTC + (q >> pb)) = __dadd_rn(W(eTC + (q >> pb)), U);
    T5 = __dadd_rn(T5, U);
  }
  // the gradient from the per-axis, per-row sums
  double vol = 1.0;
  for (int k = 0; k < d; ++k) {
    double c, h;
    ch(k, c, h);
    vol = __dmul_rn(vol, __dmul_rn(2.0, h));
  }
  for (int j = 0; j < d; ++j) {
    double c, h;
    ch(j, c, h);
    // sum of w D over the sign patterns with bit j set (-lambda5 on axis j)
    double hm5 = 0.0;
    if (j < pa) {
      for (int t = 0; t < nlo; ++t)
        if ((t >> j) & 1) hm5 = __dadd_rn(hm5, W(eTL + t));
    } else if (j < pa + pb) {
      for (int t = 0; t < (1 << pb); ++t)
        if ((t >> (j - pa)) & 1) hm5 = __dadd_rn(hm5, W(eTB + t));
    } else {
      for (int t = 0; t < (1 << pc); ++t)
        if ((t >> (j - pa - pb)) & 1) hm5 = __dadd_rn(hm5, W(eTC + t));
    }
    const double a0 = W(eHA + 4 * j), a1 = W(eHA + 4 * j + 1);
    const double a2 = W(eHA + 4 * j + 2), a3 = W(eHA + 4 * j + 3);
    const double g0 = W(eG4 + 2 * j), g1 = W(eG4 + 2 * j + 1);
    double Hr[7];
    Hr[kXC] = __dadd_rn(__dadd_rn(hC, __dsub_rn(T23, __dadd_rn(__dadd_rn(a0, a1),
                                                                 __dadd_rn(a2, a3)))),
                        __dsub_rn(T4, __dadd_rn(g0, g1)));
    Hr[kXP2] = a0;
    Hr[kXM2] = a1;
    Hr[kXP3] = __dadd_rn(a2, g0);
    Hr[kXM3] = __dadd_rn(a3, g1);
    Hr[kXP5] = __dsub_rn(T5, hm5);
    Hr[kXM5] = hm5;
    double ga = 0.0, gu = 0.0;
#pragma unroll
    for (int row = 0; row < 7; ++row) {
      const double lam = row == kXC ? 0.0
                         : row == kXP2 ? lam2 : row == kXM2 ? -lam2
                         : row == kXP3 ? lam3 : row == kXM3 ? -lam3
                         : row == kXP5 ? lam5 : -lam5;
      const double x = row == kXC ? c : fma(lam, h, c);
      double ca, cu;
      SG::coef(*P, j, x, ca, cu);
      ga = fma(Hr[row], ca, ga);
      gu = fma(Hr[row], cu, gu);
    }
    if constexpr (FAM == GMQ_OSCILLATORY) {
      // base 2 pi u_1: dS/du_1 = 2 pi at every node
      if (j == 0)
        gu = fma(2.0 * M_PI, __dadd_rn(__dadd_rn(hC, T23), __dadd_rn(T4, T5)), gu);
    }
    A.out[(int64_t)j * A.ldo + r] = __dmul_rn(vol, ga);
    A.out[(int64_t)(d + j) * A.ldo + r] = __dmul_rn(vol, gu);
  }
  double t7 = __dmul_rn(w7[0], s1);
  t7 = fma(w7[1], s2, t7);
  t7 = fma(w7[2], s3, t7);
  t7 = fma(w7[3], s4, t7);
  t7 = fma(w7[4], s5, t7);
  A.out[(int64_t)(2 * d) * A.ldo + r] = __dmul_rn(vol, t7);
}

template <int FAM>
cudaError_t launch_rule_grad_sep(const GradArgs& A, cudaStream_t s) {
  const size_t smem = grad_sep_smem_bytes(A.P.d, Sep<FAM>::kFlag);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rule_grad_sep<FAM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (A.n + kGradSepBlock - 1) / kGradSepBlock;
  if (blocks == 0) return cudaSuccess;
  k_rule_grad_sep<FAM><<<(unsigned)blocks, kGradSepBlock, smem, s>>>(A);
  return cudaGetLastError();
}

constexpr int kGradBlock = 64;

inline size_t grad_smem_bytes(int d) {
  return sizeof(double) * ((size_t)2 * d * kGradBlock            // centres, half-widths
                           + (size_t)kXRows * d * kGradBlock     // node coordinates
                           + (size_t)2 * d * kGradBlock)         // gradient accumulators
         + sizeof(SmemParams<double>) + 16;
}

template <int FAM>
__global__ void __launch_bounds__(kGradBlock) k_rule_grad(const GradArgs A) {
  constexpr int RB = kGradBlock;
  extern __shared__ __align__(16) double smem[];
  const int d = A.P.d;
  double* cd = smem;
  double* hd = cd + d * RB;
  double* xt = hd + d * RB;
  double* acc = xt + kXRows * d * RB;  // [2d][RB]
  SmemParams<double>* P = reinterpret_cast<SmemParams<double>*>(acc + 2 * d * RB);
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int j = tid; j < d; j += RB) {
    P->a[j] = A.P.a[j];
    P->u[j] = A.P.u[j];
    P->b[j] = A.P.b[j];
  }
  if (tid == 0) P->c0 = A.P.c0;
  const double l2 = A.R.lam2, l3 = A.R.lam3, l5 = A.R.lam5;
  for (int idx = tid; idx < d * RB; idx += RB) {
    const int k = idx / RB, q = idx - k * RB;
    const int64_t r = r0 + q;
    double cv = 0.5, hv = 0.25;
    if (r < A.n) {
      cv = A.c[(int64_t)k * A.ld + r];
      hv = A.h[(int64_t)k * A.ld + r];
    }
    cd[k * RB + q] = cv;
    hd[k * RB + q] = hv;
    xt[(kXC * d + k) * RB + q] = cv;
    xt[(kXP2 * d + k) * RB + q] = fma(l2, hv, cv);
    xt[(kXM2 * d + k) * RB + q] = fma(-l2, hv, cv);
    xt[(kXP3 * d + k) * RB + q] = fma(l3, hv, cv);
    xt[(kXM3 * d + k) * RB + q] = fma(-l3, hv, cv);
    xt[(kXP5 * d + k) * RB + q] = fma(l5, hv, cv);
    xt[(kXM5 * d + k) * RB + q] = fma(-l5, hv, cv);
  }
  for (int idx = tid; idx < 2 * d * RB; idx += RB) acc[idx] = 0.0;
  __syncthreads();
  const int64_t r = r0 + tid;
  if (r >= A.n) return;
  const int N = (int)A.R.nodes;
  const int b4 = 1 + 4 * d, b5 = b4 + 2 * d * (d - 1);
  double* ga = acc + tid;
  double* gu = acc + d * RB + tid;
  double S = 0.0;
  int pj = 0, pk = 1, pcount = 0;  // running (j, k) of the pair class
  for (int i = 0; i < N; ++i) {
    int kind, k1 = -1, r1 = kXC, k2 = -1, r2 = kXC;
    unsigned m = 0u;
    if (i == 0) {
      kind = 0;
    } else if (i < b4) {
      const int q = i - 1;
      k1 = q >> 2;
      r1 = kXP2 + (q & 3);
      kind = (q & 3) < 2 ? 1 : 2;
    } else if (i < b5) {
      const int q = i - b4;
      k1 = pj;
      k2 = pk;
      r1 = (q & 2) ? kXM3 : kXP3;
      r2 = (q & 1) ? kXM3 : kXP3;
      kind = 3;
      if (++pcount == 4) {  // next pair in (j, k) lexicographic order
        pcount = 0;
        if (++pk == d) {
          ++pj;
          pk = pj + 1;
        }
      }
    } else {
      m = (unsigned)(i - b5);
      kind = 4;
    }
    auto X = [&](int j) -> double {
      int row;
      if (kind == 4)
        row = ((m >> j) & 1u) ? kXM5 : kXP5;
      else
        row = (j == k1) ? r1 : ((j == k2) ? r2 : kXC);
      return xt[(row * d + j) * RB + tid];
    };
    const double w = A.R.w7[kind];
    S = fma(w, FamilyGrad<FAM>::eval(*P, d, X, w, ga, gu, RB), S);
  }
  double vol = 1.0;
  for (int k = 0; k < d; ++k) vol = vol * (2.0 * hd[k * RB + tid]);
  for (int j = 0; j < d; ++j) {
    A.out[(int64_t)j * A.ldo + r] = vol * ga[j * RB];
    A.out[(int64_t)(d + j) * A.ldo + r] = vol * gu[j * RB];
  }
  A.out[(int64_t)(2 * d) * A.ldo + r] = vol * S;
}

template <int FAM>
cudaError_t launch_rule_grad_family(const GradArgs& A, cudaStream_t s) {
  if (!A.nodewise) return launch_rule_grad_sep<FAM>(A, s);
  const size_t smem = grad_smem_bytes(A.P.d);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rule_grad<FAM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (A.n + kGradBlock - 1) / kGradBlock;
  if (blocks == 0) return cudaSuccess;
  k_rule_grad<FAM><<<(unsigned)blocks, kGradBlock, smem, s>>>(A);
  return cudaGetLastError();
}

#define GMQ_DEFINE_GRAD_FAMILY(FAMV)                                                   \
  template cudaError_t launch_rule_grad_family<FAMV>(const GradArgs& A, cudaStream_t s);

}  // namespace gmq
