// gmq_families.cuh -- built-in integrands as device functors (paper Sec. 4
// test functions; Genz families).  Each functor evaluates f at one node
// whose coordinates it reads through an accessor x(j), j = 0..d-1, so the
// rule kernel never materialises the node vector.  Per-family constants
// (a_j^2, a_j^-2, 2 pi u_1) are precomputed once per problem on the host.
#pragma once

#include "gmq_common.cuh"

namespace gmq {

// Parameters staged in shared memory by the rule kernel.
struct SmemParams {
  double a[GMQ_MAX_DIM];
  double u[GMQ_MAX_DIM];
  double b[GMQ_MAX_DIM];
  double c0;
};

// x^e for a positive integer exponent by binary powering.
__device__ __forceinline__ double ipow(double x, int e) {
  double r = 1.0;
  while (e) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

__device__ __forceinline__ float ipowf(float x, int e) {
  float r = 1.0f;
  while (e) {
    if (e & 1) r *= x;
    x *= x;
    e >>= 1;
  }
  return r;
}

template <int FAM>
struct Family;

// cos(2 pi u_1 + sum a_j x_j)
template <>
struct Family<GMQ_OSCILLATORY> {
  template <class X>
  __device__ __forceinline__ static double eval(const SmemParams& P, int d, X x) {
    double s = P.c0;
    for (int j = 0; j < d; ++j) s = fma(P.a[j], x(j), s);
    return cos(s);
  }
};

// prod_j 1/(a_j^-2 + (x_j - u_j)^2), evaluated as one reciprocal of the
// product of the denominators (b_j = a_j^-2)
template <>
struct Family<GMQ_PRODUCT_PEAK> {
  template <class X>
  __device__ __forceinline__ static double eval(const SmemParams& P, int d, X x) {
    double den = 1.0;
    for (int j = 0; j < d; ++j) {
      double t = x(j) - P.u[j];
      den *= fma(t, t, P.b[j]);
    }
    return 1.0 / den;
  }
};

// (1 + sum a_j x_j)^-(d+1)
template <>
struct Family<GMQ_CORNER_PEAK> {
  template <class X>
  __device__ __forceinline__ static double eval(const SmemParams& P, int d, X x) {
    double s = 1.0;
    for (int j = 0; j < d; ++j) s = fma(P.a[j], x(j), s);
    return 1.0 / ipow(s, d + 1);
  }
};

// exp(-sum a_j^2 (x_j - u_j)^2)  (b_j = a_j^2)
template <>
struct Family<GMQ_GAUSSIAN> {
  template <class X>
  __device__ __forceinline__ static double eval(const SmemParams& P, int d, X x) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
      double t = x(j) - P.u[j];
      s = fma(P.b[j], t * t, s);
    }
    return exp(-s);
  }
};

// exp(-sum a_j |x_j - u_j|)
template <>
struct Family<GMQ_C0> {
  template <class X>
  __device__ __forceinline__ static double eval(const SmemParams& P, int d, X x) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) s = fma(P.a[j], fabs(x(j) - P.u[j]), s);
    return exp(-s);
  }
};

// 0 if any x_j > u_j, else exp(sum a_j x_j)
template <>
struct Family<GMQ_DISCONTINUOUS> {
  template <class X>
  __device__ __forceinline__ static double eval(const SmemParams& P, int d, X x) {
    double s = 0.0;
    bool zero = false;
    for (int j = 0; j < d; ++j) {
      double xj = x(j);
      zero = zero || (xj > P.u[j]);
      s = fma(P.a[j], xj, s);
    }
    return zero ? 0.0 : exp(s);
  }
};

// (sum x_j^2)^11
template <>
struct Family<GMQ_POLY_SUMSQ11> {
  template <class X>
  __device__ __forceinline__ static double eval(const SmemParams& P, int d, X x) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
      double xj = x(j);
      s = fma(xj, xj, s);
    }
    double s2 = s * s, s4 = s2 * s2, s8 = s4 * s4;
    return s8 * s2 * s;
  }
};

}  // namespace gmq
