// gmq_families.cuh -- built-in integrands as device functors (paper Sec. 4
// test functions; Genz families).  Each functor evaluates f at one node
// whose coordinates it reads through an accessor x(j), j = 0..d-1, so the
// rule kernel never materialises the node vector.  Per-family constants
// (a_j^2, a_j^-2, 2 pi u_1) are precomputed once per problem on the host.
// Real = double is the FP64 path; Real = float the mixed path's integrand.
#pragma once

#include "gm_math_tables.cuh"
#include "gmq_common.cuh"

namespace gmq {

// Parameters staged in shared memory by the rule kernel.
template <class Real>
struct SmemParams {
  Real a[GMQ_MAX_DIM];
  Real u[GMQ_MAX_DIM];
  Real b[GMQ_MAX_DIM];
  Real c0;
};

// FP64 exponential by Tang's table-driven method (P. T. P. Tang, ACM TOMS
// 15(2), 1989): x = (256 m + j) ln2/256 + r with |r| <= ln2/512, so exp(x) =
// 2^m 2^(j/256) exp(r); exp(r) - 1 is its Taylor polynomial of degree 4
// (truncation below 3.8e-17), 2^(j/256) comes from a 256-entry table and 2^m
// is added to the exponent field.  Nine FP64 instructions (the library exp
// measured ~16.6 in the rule kernels), within about one ulp of the exact
// value (gm_math_tables.cuh holds the constants, computed in 60-digit
// decimal arithmetic).  |x| >= 512 (which covers the overflow and subnormal
// ranges) and NaN go to the library exp.
__device__ __forceinline__ double gm_exp(double x) {
  // |x| < 512, tested on the high word (no FP64 compare)
  if (((unsigned)__double2hiint(x) & 0x7fffffffu) >= 0x40800000u) return exp(x);
  const double shifter = 6755399441055744.0;  // 1.5 * 2^52: low word of t = nearest integer
  const double t = fma(x, kExpInvL, shifter);
  const int n = __double2loint(t);            // round(x * 256 / ln2)
  const double nd = __dsub_rn(t, shifter);    // the same integer as a double (exact)
  double r = fma(-nd, kExpL1, x);             // exact (fused: x - n L1 fits 53 bits)
  r = fma(-nd, kExpL2, r);
  double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  q = fma(q, r, 1.0);
  const double em1 = __dmul_rn(q, r);         // exp(r) - 1
  const double T = __ldg(&kExp2Tab[n & ((1 << kExpTabBits) - 1)]);
  const double y = fma(T, em1, T);            // 2^(j/256) exp(r), in [2^(-1/512), 2^(511/512)]
  const unsigned hi = (unsigned)__double2hiint(y) + ((unsigned)(n >> kExpTabBits) << 20);
  return __hiloint2double((int)hi, __double2loint(y));
}

__device__ __forceinline__ double gexp(double x) { return gm_exp(x); }

// FP64 reciprocal: the hardware's approximate reciprocal (PTX
// rcp.approx.ftz.f64, relative error about 2^-23) refined by two
// Newton-Raphson steps y <- y + y (1 - x y) (P. Markstein, IBM J. Res. Dev.
// 34(1), 1990), each of which doubles the number of correct bits: within one
// ulp of 1/x for 2^-120 <= |x| <= 2^120, at four FP64 FMAs.  Other inputs
// (near the ends of the range, 0, inf, NaN) take the library's division.
__device__ __forceinline__ double gm_rcp(double x) {
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;  // biased exponent
  if (ex - (1023u - 120u) > 240u) return 1.0 / x;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float grcp(float x) { return 1.0f / x; }
__device__ __forceinline__ double grcp(double x) { return gm_rcp(x); }
__device__ __forceinline__ float gexp(float x) { return expf(x); }
// FP64 cosine by the same table-driven scheme (J.-M. Muller, Elementary
// Functions, ch. 6): x = n pi/128 + r with a two-part Cody-Waite reduction
// (with fused multiply-adds the first part's step is exact and the second's
// error is below 2^-70 for |x| < 2^16), |r| <= pi/256; cos(x) = C_j cos(r) -
// S_j sin(r), j = n mod 256, with C_j = cos(j pi/128), S_j = sin(j pi/128)
// from 256-entry tables, cos(r) - 1 and sin(r) by their Taylor polynomials of
// degree 6 and 5 (truncation below 1e-17).  Thirteen FP64 instructions;
// absolute error within a few units of 2^-53.  |x| >= 2^16 and non-finite x:
// the library cos.
__device__ __forceinline__ double gm_cos(double x) {
  // |x| < 2^16, tested on the high word (no FP64 compare)
  if (((unsigned)__double2hiint(x) & 0x7fffffffu) >= 0x40f00000u) return cos(x);
  const double shifter = 6755399441055744.0;  // 1.5 * 2^52
  const double t = fma(x, kCosInvQ, shifter);
  const int n = __double2loint(t);            // round(x * 128 / pi)
  const double nd = __dsub_rn(t, shifter);
  double r = fma(-nd, kCosP1, x);             // exact
  r = fma(-nd, kCosP2, r);
  const double z = __dmul_rn(r, r);
  double c = fma(z, -1.0 / 720.0, 1.0 / 24.0);
  c = fma(c, z, -0.5);
  const double cm1 = __dmul_rn(c, z);         // cos(r) - 1
  const double sp = fma(z, 1.0 / 120.0, -1.0 / 6.0);
  const double sr = fma(__dmul_rn(r, z), sp, r);  // sin(r)
  const int j = n & ((1 << kCosTabBits) - 1);
  const double C = __ldg(&kCosTab[j]), S = __ldg(&kSinTab[j]);
  return fma(-S, sr, fma(C, cm1, C));
}
__device__ __forceinline__ double gcos(double x) { return gm_cos(x); }
__device__ __forceinline__ float gcos(float x) { return cosf(x); }

// x^e for an integer exponent e >= 1 by binary powering: the low zero bits
// of e square x, the lowest one bit starts the product, each higher bit
// squares once more and multiplies in the set ones (x^9: three squarings
// and one product).
template <class Real>
__device__ __forceinline__ Real ipow(Real x, int e) {
  if (e < 1) return Real(1);
  while (!(e & 1)) {
    x *= x;
    e >>= 1;
  }
  Real r = x;
  while (e >>= 1) {
    x *= x;
    if (e & 1) r *= x;
  }
  return r;
}

template <int FAM>
struct Family;

// cos(2 pi u_1 + sum a_j x_j)
template <>
struct Family<GMQ_OSCILLATORY> {
  template <class Real, class PT, class X>
  __device__ __forceinline__ static Real eval(const PT& P, int d, X x) {
    Real s = P.c0;
#pragma unroll
    for (int j = 0; j < d; ++j) s = fma(P.a[j], x(j), s);
    return gcos(s);
  }
};

// prod_j 1/(a_j^-2 + (x_j - u_j)^2), evaluated as one reciprocal of the
// product of the denominators (b_j = a_j^-2)
template <>
struct Family<GMQ_PRODUCT_PEAK> {
  template <class Real, class PT, class X>
  __device__ __forceinline__ static Real eval(const PT& P, int d, X x) {
    Real den = Real(1);
#pragma unroll
    for (int j = 0; j < d; ++j) {
      Real t = x(j) - P.u[j];
      den *= fma(t, t, P.b[j]);
    }
    return grcp(den);
  }
};

// (1 + sum a_j x_j)^-(d+1)
template <>
struct Family<GMQ_CORNER_PEAK> {
  template <class Real, class PT, class X>
  __device__ __forceinline__ static Real eval(const PT& P, int d, X x) {
    Real s = Real(1);
#pragma unroll
    for (int j = 0; j < d; ++j) s = fma(P.a[j], x(j), s);
    return grcp(ipow(s, d + 1));
  }
};

// exp(-sum a_j^2 (x_j - u_j)^2)  (b_j = a_j^2)
template <>
struct Family<GMQ_GAUSSIAN> {
  template <class Real, class PT, class X>
  __device__ __forceinline__ static Real eval(const PT& P, int d, X x) {
    Real s = Real(0);
#pragma unroll
    for (int j = 0; j < d; ++j) {
      Real t = x(j) - P.u[j];
      s = fma(P.b[j], t * t, s);
    }
    return gexp(-s);
  }
};

// exp(-sum a_j |x_j - u_j|)
template <>
struct Family<GMQ_C0> {
  template <class Real, class PT, class X>
  __device__ __forceinline__ static Real eval(const PT& P, int d, X x) {
    Real s = Real(0);
#pragma unroll
    for (int j = 0; j < d; ++j) s = fma(P.a[j], fabs(x(j) - P.u[j]), s);
    return gexp(-s);
  }
};

// 0 if any x_j > u_j, else exp(sum a_j x_j)
template <>
struct Family<GMQ_DISCONTINUOUS> {
  template <class Real, class PT, class X>
  __device__ __forceinline__ static Real eval(const PT& P, int d, X x) {
    Real s = Real(0);
    bool zero = false;
#pragma unroll
    for (int j = 0; j < d; ++j) {
      Real xj = x(j);
      zero = zero || (xj > P.u[j]);
      s = fma(P.a[j], xj, s);
    }
    return zero ? Real(0) : gexp(s);
  }
};

// (sum x_j^2)^11
template <>
struct Family<GMQ_POLY_SUMSQ11> {
  template <class Real, class PT, class X>
  __device__ __forceinline__ static Real eval(const PT& P, int d, X x) {
    Real s = Real(0);
#pragma unroll
    for (int j = 0; j < d; ++j) {
      Real xj = x(j);
      s = fma(xj, xj, s);
    }
    Real s2 = s * s, s4 = s2 * s2, s8 = s4 * s4;
    return s8 * s2 * s;
  }
};

// Class-sum accumulators: plain FP64 sums, or FP32 sums compensated with
// Knuth's TwoSum (the rounding error of every addition is carried in c).
template <class Real>
struct Acc;

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct Acc<float> {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float ap = __fsub_rn(t, bp);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, ap), __fsub_rn(v, bp)));
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace gmq
