// gm_adjoint.cuh -- adjoint of the rule over a frozen partition.
//
// For a fixed set of regions (the leaves an adaptive integration ended
// with), the quadrature value is Q(theta) = sum_r vol_r sum_i w_i f(x_i;
// theta), with the degree-7 Genz-Malik weights w_i of the node's class.
// Its exact gradient with respect to the integrand parameters theta =
// (a_1..a_d, u_1..u_d) is the same rule applied to df/dtheta:
//   dQ/dtheta_k = sum_r vol_r sum_i w_i df/dtheta_k(x_i).
// k_rule_grad evaluates f and its 2d parameter derivatives at every node
// (thread per region, node coordinates from the same shared-memory table as
// the rule kernel), accumulates w_i * df/dtheta_k per region and writes the
// region's contributions (and its I7) to a [2d+1][n] array; the per-row
// pairwise-tree sums give Q and its gradient.
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
