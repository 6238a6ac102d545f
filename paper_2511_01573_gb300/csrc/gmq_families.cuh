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

// The integer n = round(x K) of a range reduction, and n as an FP64 value,
// without FP64 instructions (the FP64 pipe issues at 1/64 of the FP32 rate):
// x is rounded to FP32 by integer operations on its bit pattern
// (round-to-nearest on the magnitude; |x| < 2^-126 gives 0), x K + 1.5 2^23
// is one FP32 fused multiply-add whose rounding to an integer leaves
// n + 2^22 in the low mantissa bits, and n is assembled into an FP64 bit
// pattern from its leading-zero count.  Valid for |x K| < 2^21; the FP32
// copy of x and of K put n within 0.5 + 2^-23 |x K| of x K, so for the
// callers' ranges (|x K| < 2^18) the reduced argument exceeds its usual
// bound by at most 3 %.
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e < 897u) return 0.0f;
  const unsigned b = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float((b + ((lo >> 28) & 1u)) | (hi & 0x80000000u));
}

__device__ __forceinline__ int round_mul_int(double x, float k) {
  const float t = __fmaf_rn(d2f_bits(x), k, 12582912.0f);  // 1.5 * 2^23
  return (int)(__float_as_uint(t) & 0x7fffffu) - 0x400000;
}

__device__ __forceinline__ double int_to_double_bits(int n) {
  if (n == 0) return 0.0;
  const unsigned a = n < 0 ? (unsigned)(-n) : (unsigned)n;
  const int lz = __clz(a);
  const unsigned m = (a << lz) << 1;  // the bits below the leading one, at the top
  const unsigned hi = (n < 0 ? 0x80000000u : 0u) | ((unsigned)(1023 + 31 - lz) << 20) | (m >> 12);
  return __hiloint2double((int)hi, (int)(m << 20));
}

// FP64 exponential by Tang's table-driven method (P. T. P. Tang, ACM TOMS
// 15(2), 1989): x = (2048 m + j) ln2/2048 + r with |r| <= ln2/4096 (up to
// 3 % more for |x| < 64, where n = 2048 m + j comes from round_mul_int), so
// exp(x) = 2^m 2^(j/2048) exp(r); exp(r) - 1 is its Taylor polynomial of
// degree 3 (truncation below 4e-17), 2^(j/2048) comes from a 2048-entry
// table (16 KB) and 2^m is added to the exponent field.  Six FP64
// instructions for |x| < 64 and eight for 64 <= |x| < 512 (the library exp
// measured ~16.6 in the rule kernels), within about one ulp of the exact
// value (gm_math_tables.cuh holds the constants, computed in 60-digit
// decimal arithmetic).  |x| >= 512 (which covers the overflow and subnormal
// ranges) and NaN go to the library exp.
__device__ __forceinline__ double gm_exp(double x) {
  // |x| < 512, tested on the high word (no FP64 compare)
  const unsigned ahi = (unsigned)__double2hiint(x) & 0x7fffffffu;
  if (ahi >= 0x40800000u) return exp(x);
  int n;
  double nd;
  if (ahi < 0x40500000u) {  // |x| < 64
    n = round_mul_int(x, (float)kExpInvL);
    nd = int_to_double_bits(n);
  } else {
    const double shifter = 6755399441055744.0;  // 1.5 * 2^52: low word of t = nearest integer
    const double t = fma(x, kExpInvL, shifter);
    n = __double2loint(t);                      // round(x * 2048 / ln2)
    nd = __dsub_rn(t, shifter);                 // the same integer as a double (exact)
  }
  double r = fma(-nd, kExpL1, x);             // exact (fused: x - n L1 fits 53 bits)
  r = fma(-nd, kExpL2, r);
  double q = fma(r, 1.0 / 6.0, 0.5);
  q = fma(q, r, 1.0);
  const double em1 = __dmul_rn(q, r);         // exp(r) - 1
  const double T = __ldg(&kExp2Tab[n & ((1 << kExpTabBits) - 1)]);
  const double y = fma(T, em1, T);            // 2^(j/2048) exp(r), in [2^(-1/2048), 2^(2049/2048)]
  const unsigned hi = (unsigned)__double2hiint(y) + ((unsigned)(n >> kExpTabBits) << 20);
  return __hiloint2double((int)hi, __double2loint(y));
}

__device__ __forceinline__ double gexp(double x) { return gm_exp(x); }

// FP64 reciprocal: the hardware's approximate reciprocal (PTX
// rcp.approx.ftz.f64, relative error about 2^-23) refined by one third-order
// step of Householder's iteration for 1/x: with e = 1 - x y (one fused
// multiply-add, exact up to its final rounding), y (1 + e + e^2) = (1/x)(1 -
// e^3), so the relative error drops from about 2^-23 to about 2^-69 before
// the last rounding: within one ulp of 1/x for 2^-120 <= |x| <= 2^120, at
// three FP64 FMAs (two Newton-Raphson steps take four).  Other inputs (near
// the ends of the range, 0, inf, NaN) take the library's division.
__device__ __forceinline__ double gm_rcp(double x) {
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;  // biased exponent
  if (ex - (1023u - 120u) > 240u) return 1.0 / x;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
// FP32 reciprocal: the correctly rounded 1/x (the bits of 1.0f / x)
__device__ __forceinline__ float grcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double grcp(double x) { return gm_rcp(x); }
__device__ __forceinline__ float gexp(float x) { return expf(x); }
// FP64 cosine by the same table-driven scheme (J.-M. Muller, Elementary
// Functions, ch. 6): x = n pi/128 + r with a two-part Cody-Waite reduction
// (with fused multiply-adds the first part's step is exact and the second's
// error is below 2^-70 for |x| < 2^16), |r| <= pi/256; cos(x) = C_j cos(r) -
// S_j sin(r), j = n mod 256, with C_j = cos(j pi/128), S_j = sin(j pi/128)
// from 256-entry tables, cos(r) - 1 and sin(r) by their Taylor polynomials of
// degree 6 and 5 (truncation below 1e-17).  Eleven FP64 instructions for
// |x| < 1024 (n from round_mul_int), thirteen above; absolute error within
// a few units of 2^-53.  |x| >= 2^16 and non-finite x:
// the library cos.
__device__ __forceinline__ double gm_cos(double x) {
  // |x| < 2^16, tested on the high word (no FP64 compare)
  const unsigned ahi = (unsigned)__double2hiint(x) & 0x7fffffffu;
  if (ahi >= 0x40f00000u) return cos(x);
  int n;
  double nd;
  if (ahi < 0x40900000u) {  // |x| < 1024: n from round_mul_int
    n = round_mul_int(x, (float)kCosInvQ);
    nd = int_to_double_bits(n);
  } else {
    const double shifter = 6755399441055744.0;  // 1.5 * 2^52
    const double t = fma(x, kCosInvQ, shifter);
    n = __double2loint(t);                      // round(x * 128 / pi)
    nd = __dsub_rn(t, shifter);
  }
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

// sin(x) and cos(x) together (the adjoint of the oscillatory family): the
// same reduction and polynomials as gm_cos, with sin(x) = S_j cos(r) +
// C_j sin(r) two more fused multiply-adds; outside the fast range the
// library's sincos.
__device__ __forceinline__ void gm_sincos(double x, double* sn, double* cs) {
  const unsigned ahi = (unsigned)__double2hiint(x) & 0x7fffffffu;
  if (ahi >= 0x40f00000u) {
    sincos(x, sn, cs);
    return;
  }
  int n;
  double nd;
  if (ahi < 0x40900000u) {
    n = round_mul_int(x, (float)kCosInvQ);
    nd = int_to_double_bits(n);
  } else {
    const double shifter = 6755399441055744.0;
    const double t = fma(x, kCosInvQ, shifter);
    n = __double2loint(t);
    nd = __dsub_rn(t, shifter);
  }
  double r = fma(-nd, kCosP1, x);
  r = fma(-nd, kCosP2, r);
  const double z = __dmul_rn(r, r);
  double c = fma(z, -1.0 / 720.0, 1.0 / 24.0);
  c = fma(c, z, -0.5);
  const double cm1 = __dmul_rn(c, z);
  const double sp = fma(z, 1.0 / 120.0, -1.0 / 6.0);
  const double sr = fma(__dmul_rn(r, z), sp, r);
  const int j = n & ((1 << kCosTabBits) - 1);
  const double C = __ldg(&kCosTab[j]), S = __ldg(&kSinTab[j]);
  *cs = fma(-S, sr, fma(C, cm1, C));
  *sn = fma(C, sr, fma(S, cm1, S));
}


// FP32 cosine of the mixed form's oscillatory integrand, by Cody and
// Waite's reduction (W. J. Cody, W. Waite, Software Manual for the
// Elementary Functions, 1980): x = n pi/2 + r, n the nearest integer to
// x 2/pi, |r| <= pi/4 (up to one rounding of the quotient), with pi/2 split
// into three FP32 parts (their sum is pi/2 to 1e-23) subtracted by fused
// multiply-adds; cos r and sin r by their Taylor polynomials of degree 8
// and 9 (truncated terms below 3e-8); the quadrant n mod 4 picks cos r,
// -sin r, -cos r or sin r.  Absolute error a few units of 2^-24 for
// |x| < 2^15; other x (and NaN) take the library cosf, outside the inlined
// path.  gm_cosf2: the same steps on two lanes with paired instructions.
static __device__ __noinline__ float gm_cosf_wide(float x) { return cosf(x); }

constexpr float kPio2A = 0x1.921fb6p+0f, kPio2B = -0x1.777a5cp-25f, kPio2C = -0x1.ee59dap-50f;
constexpr float kTwoOverPi = 0.636619747f;

__device__ __forceinline__ float cosf_quadrant(float c, float s, int q) {
  const float v = (q & 1) ? s : c;
  return ((q + 1) & 2) ? -v : v;
}

__device__ __forceinline__ float gm_cosf(float x) {
  if (!(fabsf(x) < 32768.0f)) return gm_cosf_wide(x);
  const float n = rintf(x * kTwoOverPi);
  float r = __fmaf_rn(-n, kPio2A, x);
  r = __fmaf_rn(-n, kPio2B, r);
  r = __fmaf_rn(-n, kPio2C, r);
  const float z = r * r;
  float c = __fmaf_rn(z, 1.0f / 40320.0f, -1.0f / 720.0f);
  c = __fmaf_rn(c, z, 1.0f / 24.0f);
  c = __fmaf_rn(c, z, -0.5f);
  c = __fmaf_rn(c, z, 1.0f);
  float sp = __fmaf_rn(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
  sp = __fmaf_rn(sp, z, 1.0f / 120.0f);
  sp = __fmaf_rn(sp, z, -1.0f / 6.0f);
  const float s = __fmaf_rn(sp, z * r, r);
  return cosf_quadrant(c, s, (int)n);
}

__device__ __forceinline__ float2 gm_cosf2(float2 x) {
  if (!(fabsf(x.x) < 32768.0f && fabsf(x.y) < 32768.0f))
    return make_float2(gm_cosf(x.x), gm_cosf(x.y));
  const float2 n = make_float2(rintf(x.x * kTwoOverPi), rintf(x.y * kTwoOverPi));
  const float2 mn = make_float2(-n.x, -n.y);
  float2 r = __ffma2_rn(mn, make_float2(kPio2A, kPio2A), x);
  r = __ffma2_rn(mn, make_float2(kPio2B, kPio2B), r);
  r = __ffma2_rn(mn, make_float2(kPio2C, kPio2C), r);
  const float2 z = __fmul2_rn(r, r);
  float2 c = __ffma2_rn(z, make_float2(1.0f / 40320.0f, 1.0f / 40320.0f),
                        make_float2(-1.0f / 720.0f, -1.0f / 720.0f));
  c = __ffma2_rn(c, z, make_float2(1.0f / 24.0f, 1.0f / 24.0f));
  c = __ffma2_rn(c, z, make_float2(-0.5f, -0.5f));
  c = __ffma2_rn(c, z, make_float2(1.0f, 1.0f));
  float2 sp = __ffma2_rn(z, make_float2(1.0f / 362880.0f, 1.0f / 362880.0f),
                         make_float2(-1.0f / 5040.0f, -1.0f / 5040.0f));
  sp = __ffma2_rn(sp, z, make_float2(1.0f / 120.0f, 1.0f / 120.0f));
  sp = __ffma2_rn(sp, z, make_float2(-1.0f / 6.0f, -1.0f / 6.0f));
  const float2 s = __ffma2_rn(sp, __fmul2_rn(z, r), r);
  return make_float2(cosf_quadrant(c.x, s.x, (int)n.x), cosf_quadrant(c.y, s.y, (int)n.y));
}

__device__ __forceinline__ float gcos(float x) { return gm_cosf(x); }

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

// Two FP32 integrand values at once.  On this GPU a paired FP32 instruction
// (FADD2 / FMUL2 / FFMA2, the __fadd2_rn / __fmul2_rn / __ffma2_rn
// intrinsics) does two lanes' adds, multiplies or fused multiply-adds in one
// issue slot, so the mixed kernels evaluate the integrand at two nodes
// together: x(j) returns the pair of the two nodes' j-th coordinates.  Each
// lane runs exactly the scalar eval's operations in the scalar eval's order
// (every paired operation rounds each lane as the scalar one does; the
// transcendental and the reciprocal run per lane), so eval2 returns the
// bits two eval calls would.
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 abs2(float2 v) { return make_float2(fabsf(v.x), fabsf(v.y)); }

template <int FAM>
struct Family2;

template <>
struct Family2<GMQ_OSCILLATORY> {
  template <class PT, class X>
  __device__ __forceinline__ static float2 eval2(const PT& P, int d, X x) {
    float2 s = bc2(P.c0);
#pragma unroll
    for (int j = 0; j < d; ++j) s = __ffma2_rn(bc2(P.a[j]), x(j), s);
    return gm_cosf2(s);
  }
};

template <>
struct Family2<GMQ_PRODUCT_PEAK> {
  template <class PT, class X>
  __device__ __forceinline__ static float2 eval2(const PT& P, int d, X x) {
    float2 den = bc2(1.0f);
#pragma unroll
    for (int j = 0; j < d; ++j) {
      const float2 t = __fadd2_rn(x(j), bc2(-P.u[j]));
      den = __fmul2_rn(den, __ffma2_rn(t, t, bc2(P.b[j])));
    }
    return make_float2(grcp(den.x), grcp(den.y));
  }
};

template <>
struct Family2<GMQ_CORNER_PEAK> {
  template <class PT, class X>
  __device__ __forceinline__ static float2 eval2(const PT& P, int d, X x) {
    float2 s = bc2(1.0f);
#pragma unroll
    for (int j = 0; j < d; ++j) s = __ffma2_rn(bc2(P.a[j]), x(j), s);
    // s^(d+1) by the binary powering of ipow, both lanes at once
    int e = d + 1;
    while (!(e & 1)) {
      s = __fmul2_rn(s, s);
      e >>= 1;
    }
    float2 r = s;
    while (e >>= 1) {
      s = __fmul2_rn(s, s);
      if (e & 1) r = __fmul2_rn(r, s);
    }
    return make_float2(grcp(r.x), grcp(r.y));
  }
};

template <>
struct Family2<GMQ_GAUSSIAN> {
  template <class PT, class X>
  __device__ __forceinline__ static float2 eval2(const PT& P, int d, X x) {
    float2 s = bc2(0.0f);
#pragma unroll
    for (int j = 0; j < d; ++j) {
      const float2 t = __fadd2_rn(x(j), bc2(-P.u[j]));
      s = __ffma2_rn(bc2(P.b[j]), __fmul2_rn(t, t), s);
    }
    return make_float2(gexp(-s.x), gexp(-s.y));
  }
};

template <>
struct Family2<GMQ_C0> {
  template <class PT, class X>
  __device__ __forceinline__ static float2 eval2(const PT& P, int d, X x) {
    float2 s = bc2(0.0f);
#pragma unroll
    for (int j = 0; j < d; ++j)
      s = __ffma2_rn(bc2(P.a[j]), abs2(__fadd2_rn(x(j), bc2(-P.u[j]))), s);
    return make_float2(gexp(-s.x), gexp(-s.y));
  }
};

template <>
struct Family2<GMQ_DISCONTINUOUS> {
  template <class PT, class X>
  __device__ __forceinline__ static float2 eval2(const PT& P, int d, X x) {
    float2 s = bc2(0.0f);
    bool zx = false, zy = false;
#pragma unroll
    for (int j = 0; j < d; ++j) {
      const float2 xj = x(j);
      zx = zx || (xj.x > P.u[j]);
      zy = zy || (xj.y > P.u[j]);
      s = __ffma2_rn(bc2(P.a[j]), xj, s);
    }
    return make_float2(zx ? 0.0f : gexp(s.x), zy ? 0.0f : gexp(s.y));
  }
};

template <>
struct Family2<GMQ_POLY_SUMSQ11> {
  template <class PT, class X>
  __device__ __forceinline__ static float2 eval2(const PT& P, int d, X x) {
    float2 s = bc2(0.0f);
#pragma unroll
    for (int j = 0; j < d; ++j) {
      const float2 xj = x(j);
      s = __ffma2_rn(xj, xj, s);
    }
    const float2 s2 = __fmul2_rn(s, s), s4 = __fmul2_rn(s2, s2), s8 = __fmul2_rn(s4, s4);
    return __fmul2_rn(__fmul2_rn(s8, s2), s);
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


// Separable form of the FP64 integrands, for the FP64 rule kernels: every
// family is f(x) = g(S) with S = base (+) phi_0(x_0) (+) ... (+)
// phi_{d-1}(x_{d-1}), where (+) is addition (kMul false) or multiplication
// (kMul true) and base, present when kBase, heads the chain.  A region's
// nodes take each coordinate from one of seven values per axis (the centre
// and c +- lambda h for the three generators), so the kernels evaluate phi
// 7 d times per region and build every node's S from per-axis terms and
// partial chains instead of d operations per node.  The discontinuous
// family also has a per-axis flag (x_j > u_j) whose OR over the axes zeroes
// f.  Every operation is rounded separately (no contraction), so a value
// does not depend on which code path or lane forms it.
template <int FAM>
struct Sep;

// cos(2 pi u_1 + sum a_j x_j)
template <>
struct Sep<GMQ_OSCILLATORY> {
  static constexpr bool kMul = false, kBase = true, kFlag = false;
  template <class PT>
  __device__ __forceinline__ static double base(const PT& P) { return P.c0; }
  template <class PT>
  __device__ __forceinline__ static double phi(const PT& P, int j, double x) {
    return __dmul_rn(P.a[j], x);
  }
  __device__ __forceinline__ static double g(int, double s) { return gcos(s); }
};

// 1 / prod_j (a_j^-2 + (x_j - u_j)^2)
template <>
struct Sep<GMQ_PRODUCT_PEAK> {
  static constexpr bool kMul = true, kBase = false, kFlag = false;
  template <class PT>
  __device__ __forceinline__ static double base(const PT&) { return 1.0; }
  template <class PT>
  __device__ __forceinline__ static double phi(const PT& P, int j, double x) {
    const double t = __dsub_rn(x, P.u[j]);
    return fma(t, t, P.b[j]);
  }
  __device__ __forceinline__ static double g(int, double s) { return grcp(s); }
};

// (1 + sum a_j x_j)^-(d+1)
template <>
struct Sep<GMQ_CORNER_PEAK> {
  static constexpr bool kMul = false, kBase = true, kFlag = false;
  template <class PT>
  __device__ __forceinline__ static double base(const PT&) { return 1.0; }
  template <class PT>
  __device__ __forceinline__ static double phi(const PT& P, int j, double x) {
    return __dmul_rn(P.a[j], x);
  }
  __device__ __forceinline__ static double g(int d, double s) { return grcp(ipow(s, d + 1)); }
};

// exp(-sum a_j^2 (x_j - u_j)^2)
template <>
struct Sep<GMQ_GAUSSIAN> {
  static constexpr bool kMul = false, kBase = false, kFlag = false;
  template <class PT>
  __device__ __forceinline__ static double base(const PT&) { return 0.0; }
  template <class PT>
  __device__ __forceinline__ static double phi(const PT& P, int j, double x) {
    const double t = __dsub_rn(x, P.u[j]);
    return __dmul_rn(P.b[j], __dmul_rn(t, t));
  }
  __device__ __forceinline__ static double g(int, double s) { return gexp(-s); }
};

// exp(-sum a_j |x_j - u_j|)
template <>
struct Sep<GMQ_C0> {
  static constexpr bool kMul = false, kBase = false, kFlag = false;
  template <class PT>
  __device__ __forceinline__ static double base(const PT&) { return 0.0; }
  template <class PT>
  __device__ __forceinline__ static double phi(const PT& P, int j, double x) {
    return __dmul_rn(P.a[j], fabs(__dsub_rn(x, P.u[j])));
  }
  __device__ __forceinline__ static double g(int, double s) { return gexp(-s); }
};

// 0 if any x_j > u_j, else exp(sum a_j x_j)
template <>
struct Sep<GMQ_DISCONTINUOUS> {
  static constexpr bool kMul = false, kBase = false, kFlag = true;
  template <class PT>
  __device__ __forceinline__ static double base(const PT&) { return 0.0; }
  template <class PT>
  __device__ __forceinline__ static double phi(const PT& P, int j, double x) {
    return __dmul_rn(P.a[j], x);
  }
  template <class PT>
  __device__ __forceinline__ static bool flag(const PT& P, int j, double x) { return x > P.u[j]; }
  __device__ __forceinline__ static double g(int, double s) { return gexp(s); }
};

// (sum x_j^2)^11
template <>
struct Sep<GMQ_POLY_SUMSQ11> {
  static constexpr bool kMul = false, kBase = false, kFlag = false;
  template <class PT>
  __device__ __forceinline__ static double base(const PT&) { return 0.0; }
  template <class PT>
  __device__ __forceinline__ static double phi(const PT&, int, double x) {
    return __dmul_rn(x, x);
  }
  __device__ __forceinline__ static double g(int, double s) {
    const double s2 = __dmul_rn(s, s), s4 = __dmul_rn(s2, s2), s8 = __dmul_rn(s4, s4);
    return __dmul_rn(__dmul_rn(s8, s2), s);
  }
};

// An FP32 value as FP64, exactly, assembled from its bit pattern with
// integer operations (the conversion instruction runs on the FP64 pipe,
// which on this GPU issues at 1/64 of the FP32 rate): sign, exponent rebased
// from 127 to 1023, the 23 fraction bits at the top of the 52.  Zero keeps
// its sign; subnormal, infinite and NaN values take the conversion.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const unsigned hi = (u & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((u >> 3) & 0xfffffu);
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}

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
  __device__ __forceinline__ double value() const { return f2d_exact(s) + f2d_exact(c); }
};

}  // namespace gmq
