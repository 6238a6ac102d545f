// gm_region32.cuh -- mixed-form evaluation of one region by one thread,
// shared by the single-integral mixed kernels (gm_rule.cuh) and the batched
// mixed kernel, so both compute a region with the same operations in the
// same order.
//
// Mixed form: node coordinates are FP32 (the caller's table, built by
// mixed_coord_rows), the integrand runs in FP32, and the class sums are
// FP32 with Knuth TwoSum compensation, converted to FP64 before the
// weights; the fourth differences and everything after the class sums are
// FP64 (region_finish64).
#pragma once

#include "gm_region64.cuh"
#include "gmq_common.cuh"
#include "gmq_families.cuh"

namespace gmq {

// The seven FP32 node-coordinate rows of one axis of a region (kXC, kXP2,
// kXM2, kXP3, kXM3, kXP5, kXM5 at out[row * stride]), formed in FP32 from
// the centre split into two FP32 parts, c = c_hi + c_lo, and the FP32
// half-width: x = c_hi + fma(+-lambda, h, c_lo).  The offset c_lo +
// lambda h is small and nearly exact, so x is c + lambda h rounded once to
// FP32 up to rare one-ulp differences -- the rounding the FP32 integrand
// sees in any case -- while the FP64 work per axis is three conversions and
// one subtraction (the FP64 pipe issues at 1/64 of the FP32 rate).
__device__ __forceinline__ void mixed_coord_rows(double c, double h, float l2, float l3,
                                                 float l5, float* out, int stride) {
  const float c_hi = __double2float_rn(c);
  const float c_lo = __double2float_rn(__dsub_rn(c, f2d_exact(c_hi)));
  const float hf = __double2float_rn(h);
  out[kXC * stride] = c_hi;
  out[kXP2 * stride] = __fadd_rn(c_hi, __fmaf_rn(l2, hf, c_lo));
  out[kXM2 * stride] = __fadd_rn(c_hi, __fmaf_rn(-l2, hf, c_lo));
  out[kXP3 * stride] = __fadd_rn(c_hi, __fmaf_rn(l3, hf, c_lo));
  out[kXM3 * stride] = __fadd_rn(c_hi, __fmaf_rn(-l3, hf, c_lo));
  out[kXP5 * stride] = __fadd_rn(c_hi, __fmaf_rn(l5, hf, c_lo));
  out[kXM5 * stride] = __fadd_rn(c_hi, __fmaf_rn(-l5, hf, c_lo));
}

// Integrand parameters in registers (compile-time dimension).
template <int D>
struct RegParams {
  float a[D], u[D], b[D];
  float c0;
};

// Generic dimension: every node in the order of its definition (centre;
// per axis +l2, -l2, +l3, -l3; pairs j < k with sign patterns ++, +-, -+,
// --; sign patterns m = 0 .. 2^d - 1).  P holds FP32 parameters;
// tab(row, j) is the FP32 node coordinate; pairs as in region_sums64.
template <int FAM, class PT, class Tab>
__device__ __forceinline__ void region_mixed_flat(const PT& P, int d, const unsigned short* pairs,
                                                  const Tab& tab, double ratio, RegionSums& o) {
  const int b4 = 1 + 4 * d;             // first pair node
  const int b5 = b4 + 2 * d * (d - 1);  // first sign-pattern node
  const int N = b5 + (1 << d);
  Acc<float> S1, S2, S3, S4, S5;
  double f0 = 0.0, two_f0 = 0.0, q0 = 0.0, q1 = 0.0, q2 = 0.0, dbest = -1.0;
  int kbest = 0;
  for (int i = 0; i < N; ++i) {
    int kind, k1 = -1, r1 = kXC, k2 = -1, r2 = kXC, w = 0;
    unsigned m = 0u;
    if (i == 0) {
      kind = 1;
    } else if (i < b4) {
      const int q = i - 1;
      k1 = q >> 2;
      w = q & 3;
      r1 = kXP2 + w;
      kind = (w < 2) ? 2 : 3;
    } else if (i < b5) {
      const int q = i - b4;
      const unsigned pr = pairs[q >> 2];
      k1 = (int)(pr >> 8);
      k2 = (int)(pr & 255u);
      r1 = (q & 2) ? kXM3 : kXP3;
      r2 = (q & 1) ? kXM3 : kXP3;
      kind = 4;
    } else {
      m = (unsigned)(i - b5);
      kind = 5;
    }
    const float v = Family<FAM>::template eval<float>(P, d, [&](int j) -> float {
      int row;
      if (kind == 5)
        row = ((m >> j) & 1u) ? kXM5 : kXP5;
      else
        row = (j == k1) ? r1 : ((j == k2) ? r2 : kXC);
      return tab(row, j);
    });
    if (kind == 5) {
      S5.add(v);
    } else if (kind == 4) {
      S4.add(v);
    } else if (kind == 1) {
      S1.add(v);
      f0 = f2d_exact(v);
      two_f0 = __dmul_rn(2.0, f0);
    } else {
      if (kind == 2)
        S2.add(v);
      else
        S3.add(v);
      const double vd = f2d_exact(v);
      if (w == 0) {
        q0 = vd;
      } else if (w == 1) {
        q1 = vd;
      } else if (w == 2) {
        q2 = vd;
      } else {
        const double t1 = __dsub_rn(__dadd_rn(q0, q1), two_f0);
        const double t2 = __dsub_rn(__dadd_rn(q2, vd), two_f0);
        const double Dk = fabs(__dsub_rn(t1, __dmul_rn(ratio, t2)));
        if (Dk > dbest) {
          dbest = Dk;
          kbest = k1;
        }
      }
    }
  }
  o.s1 = S1.value();
  o.s2 = S2.value();
  o.s3 = S3.value();
  o.s4 = S4.value();
  o.s5 = S5.value();
  o.f0 = f0;
  o.dbest = dbest;
  o.kbest = kbest;
}

// Dimension D known at compile time (3 <= D <= 16).  Every node is
// evaluated together with its partner in one paired FP32 evaluation
// (Family2::eval2), the partner being the node that differs from it in one
// coordinate only: the two signs of +-lambda2 e_k and of +-lambda3 e_k; for
// a pair j < k, the two signs on axis k with the same sign on axis j; in the
// sign-pattern class, the two signs on axis 0.  The nodes of classes 1-4 are
// formed from the centre held in registers and the one or two coordinates
// they move (read from the table), with the moved axis k known at compile
// time (unrolled over k, the pair's first axis j in a loop).  The 2^D
// sign-pattern nodes are walked in Gray-code order over a register-resident
// node vector: consecutive patterns differ in one coordinate, which moves
// between c_k + l5 h_k and c_k - l5 h_k by XOR-ing the two FP32 bit
// patterns.  In an aligned group of eight patterns the coordinates that
// change are axes 0, 1, 0, 2, 0, 1, 0, so the group is four axis-0 pairs,
// with axes 1, 2, 1 stepping between them; the axis changed on entering the
// group (>= 3) is picked with a predicated select.  Every class sum adds its
// node values one by one in definition order (Gray-code order for the last
// class), as the one-node-at-a-time walk did.  Pf holds the FP32 parameters
// (read once into registers).
template <int FAM, int D, class PT, class Tab>
__device__ __forceinline__ void region_mixed_walk(const PT& Pf, const Tab& tab, double ratio,
                                                  RegionSums& o) {
  static_assert(D >= 3 && D <= 16, "the Gray walk needs D >= 3");
  RegParams<D> rp;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    rp.a[j] = Pf.a[j];
    rp.u[j] = Pf.u[j];
    rp.b[j] = Pf.b[j];
  }
  rp.c0 = Pf.c0;
  Acc<float> S1, S2, S3, S4, S5;
  double dbest = -1.0;
  int kbest = 0;
  float xc[D];
#pragma unroll
  for (int j = 0; j < D; ++j) xc[j] = tab(kXC, j);
  // class 1: the centre
  const float vc = Family<FAM>::template eval<float>(rp, D, [&](int j) -> float { return xc[j]; });
  S1.add(vc);
  const double f0 = f2d_exact(vc);
  const double two_f0 = __dmul_rn(2.0, f0);
  // classes 2 and 3: per axis k the pairs (+l2, -l2) and (+l3, -l3), and
  // the fourth difference of axis k
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float2 p2 = make_float2(tab(kXP2, k), tab(kXM2, k));
    const float2 p3 = make_float2(tab(kXP3, k), tab(kXM3, k));
    const float2 v2 = Family2<FAM>::eval2(
        rp, D, [&](int j) -> float2 { return j == k ? p2 : bc2(xc[j]); });
    const float2 v3 = Family2<FAM>::eval2(
        rp, D, [&](int j) -> float2 { return j == k ? p3 : bc2(xc[j]); });
    S2.add(v2.x);
    S2.add(v2.y);
    S3.add(v3.x);
    S3.add(v3.y);
    const double t1 = __dsub_rn(__dadd_rn(f2d_exact(v2.x), f2d_exact(v2.y)), two_f0);
    const double t2 = __dsub_rn(__dadd_rn(f2d_exact(v3.x), f2d_exact(v3.y)), two_f0);
    const double Dk = fabs(__dsub_rn(t1, __dmul_rn(ratio, t2)));
    if (Dk > dbest) {
      dbest = Dk;
      kbest = k;
    }
  }
  // class 4: pairs j < k, sign patterns ++, +-, -+, -- (the pairs on axis k)
  for (int j = 0; j < D - 1; ++j) {
    const float pj = tab(kXP3, j), mj = tab(kXM3, j);
#pragma unroll
    for (int k = 1; k < D; ++k) {
      if (k > j) {
        const float2 pk = make_float2(tab(kXP3, k), tab(kXM3, k));
        const float2 va = Family2<FAM>::eval2(rp, D, [&](int i) -> float2 {
          return i == k ? pk : bc2(i == j ? pj : xc[i]);
        });
        const float2 vb = Family2<FAM>::eval2(rp, D, [&](int i) -> float2 {
          return i == k ? pk : bc2(i == j ? mj : xc[i]);
        });
        S4.add(va.x);
        S4.add(va.y);
        S4.add(vb.x);
        S4.add(vb.y);
      }
    }
  }
  // class 5: Gray-code walk over the 2^D sign patterns in registers
  float x[D];
  unsigned tog[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float p5 = tab(kXP5, k), m5 = tab(kXM5, k);
    x[k] = p5;
    tog[k] = __float_as_uint(p5) ^ __float_as_uint(m5);
  }
  auto flip = [&](int k) { x[k] = __uint_as_float(__float_as_uint(x[k]) ^ tog[k]); };
  // the pattern x and its axis-0 partner, in walk order
  auto pair5 = [&]() {
    const float2 x0 = make_float2(x[0], __uint_as_float(__float_as_uint(x[0]) ^ tog[0]));
    const float2 v = Family2<FAM>::eval2(rp, D, [&](int i) -> float2 {
      return i == 0 ? x0 : bc2(x[i]);
    });
    S5.add(v.x);
    S5.add(v.y);
  };
  for (unsigned tb = 0; tb < (1u << D); tb += 8u) {
    if (tb) {
      const int jb = __ffs(tb) - 1;
#pragma unroll
      for (int k = 3; k < D; ++k)
        if (k == jb) flip(k);
    }
    pair5();  // patterns 0, 1 of the group
    flip(0);
    flip(1);
    pair5();  // 2, 3
    flip(0);
    flip(2);
    pair5();  // 4, 5
    flip(0);
    flip(1);
    pair5();  // 6, 7
    flip(0);  // the group ends on pattern 7
  }
  o.s1 = S1.value();
  o.s2 = S2.value();
  o.s3 = S3.value();
  o.s4 = S4.value();
  o.s5 = S5.value();
  o.f0 = f0;
  o.dbest = dbest;
  o.kbest = kbest;
}

}  // namespace gmq
