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

// Dimension D known at compile time (3 <= D <= 16), one thread per region,
// everything in registers.  The integrand's separable form (SepF<FAM>: f =
// g(S), S = base (+) phi_0(x_0) (+) ... (+) phi_{D-1}(x_{D-1})) is used as
// in the FP64 kernels: phi at the 7 D coordinate values of the region once,
// and each node's S from one combine of per-axis terms and partial chains
// (FP32):
//   centre            S = base (+) suf_0;  suf_k = phi_k(c) (+) suf_{k+1}
//   axis node k       S = (pre_k (+) phi_k(x)) (+) suf_{k+1};
//                     pre_k = base (+) phi_0(c) (+) ... (+) phi_{k-1}(c)
//   pair node j < k   S = ((pre_j (+) phi_j(x_j)) (+) mid_jk) (+)
//                         (phi_k(x_k) (+) suf_{k+1})
//   class-5 node m    S = A[m_A] (+) (B[m_B] (+) C[m_C]) over the axis
//                     groups [0, 4), [4, 8), [8, D) (fewer for small D).
// Every node is evaluated together with its partner (paired FP32
// instructions: g2, and the last combine), the partner being the node that
// differs from it in one coordinate only: the two signs of +-lambda2 e_k
// and of +-lambda3 e_k; for a pair j < k, the two signs on axis k with the
// same sign on axis j; in the last class, the two signs on axis 0.  The
// class sums add the node values one by one in definition order (sign
// patterns in ascending order, even and odd patterns in two accumulators).
// Loops whose bodies hold the integrand run over the pair's first axis and
// over the sign-pattern blocks at run time, which keeps the kernel's code
// small enough for the instruction cache.  Pf holds the FP32 parameters (read once
// into registers); tab(row, j) is the FP32 node coordinate.
template <int FAM, int D, class PT, class Tab>
__device__ __forceinline__ void region_mixed_walk(const PT& Pf, const Tab& tab, double ratio,
                                                  RegionSums& o) {
  static_assert(D >= 3 && D <= 16, "the register walk needs D >= 3");
  using SF = SepF<FAM>;
  constexpr bool kMul = Sep<FAM>::kMul, kBase = Sep<FAM>::kBase, kFlag = Sep<FAM>::kFlag;
  RegParams<D> rp;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    rp.a[j] = Pf.a[j];
    rp.u[j] = Pf.u[j];
    rp.b[j] = Pf.b[j];
  }
  rp.c0 = Pf.c0;
  auto op = [](float x, float y) -> float {
    if constexpr (kMul)
      return __fmul_rn(x, y);
    else
      return __fadd_rn(x, y);
  };
  auto op2 = [](float2 x, float2 y) -> float2 {
    if constexpr (kMul)
      return __fmul2_rn(x, y);
    else
      return __fadd2_rn(x, y);
  };
  // discontinuous family: flag bits (x_j > u_j) of the centre, of
  // c +- lambda3 h (+ in bits 0..15, - in 16..31) and of c +- lambda5 h
  unsigned zc = 0u, z3 = 0u, z5 = 0u;
  auto g2z = [&](float2 S, bool zx, bool zy) -> float2 {
    float2 v = SF::g2(D, S);
    if constexpr (kFlag) {
      if (zx) v.x = 0.0f;
      if (zy) v.y = 0.0f;
    }
    return v;
  };
  Acc<float> S1, S2, S3, S4, S5;
  double dbest = -1.0;
  int kbest = 0;
  float fc[D], suf[D];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    const float xc = tab(kXC, j);
    fc[j] = SF::phi(rp, j, xc);
    if constexpr (kFlag) zc |= (unsigned)SF::flag(rp, j, xc) << j;
  }
  suf[D - 1] = fc[D - 1];
#pragma unroll
  for (int k = D - 2; k >= 0; --k) suf[k] = op(fc[k], suf[k + 1]);
  // class 1: the centre
  {
    const float sc = kBase ? op(SF::base(rp), suf[0]) : suf[0];
    const float vc = g2z(make_float2(sc, sc), zc != 0u, zc != 0u).x;
    S1.add(vc);
    o.f0 = f2d_exact(vc);
  }
  const double two_f0 = __dmul_rn(2.0, o.f0);
  // classes 2 and 3: per axis k the pairs (+l2, -l2) and (+l3, -l3), the
  // fourth difference of axis k, and the pair-node prefixes L3 and
  // suffixes R3 of the +-lambda3 values
  float2 L3[D], R3[D];
  float pre = kBase ? SF::base(rp) : 0.0f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const bool hp = k > 0 || kBase;
    const float2 x2 = make_float2(tab(kXP2, k), tab(kXM2, k));
    const float2 x3 = make_float2(tab(kXP3, k), tab(kXM3, k));
    const float2 ph2 = SF::phi2(rp, k, x2), ph3 = SF::phi2(rp, k, x3);
    const float2 lp2 = hp ? op2(bc2(pre), ph2) : ph2;
    const float2 lp3 = hp ? op2(bc2(pre), ph3) : ph3;
    L3[k] = lp3;
    R3[k] = k < D - 1 ? op2(ph3, bc2(suf[k + 1])) : ph3;
    const float2 s2 = k < D - 1 ? op2(lp2, bc2(suf[k + 1])) : lp2;
    const float2 s3 = k < D - 1 ? op2(lp3, bc2(suf[k + 1])) : lp3;
    bool z2x = false, z2y = false, z3x = false, z3y = false;
    if constexpr (kFlag) {
      const bool zo = (zc & ~(1u << k)) != 0u;
      const bool fp3 = SF::flag(rp, k, x3.x), fm3 = SF::flag(rp, k, x3.y);
      z3 |= ((unsigned)fp3 << k) | ((unsigned)fm3 << (k + 16));
      z2x = zo || SF::flag(rp, k, x2.x);
      z2y = zo || SF::flag(rp, k, x2.y);
      z3x = zo || fp3;
      z3y = zo || fm3;
    }
    const float2 v2 = g2z(s2, z2x, z2y);
    const float2 v3 = g2z(s3, z3x, z3y);
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
    pre = hp ? op(pre, fc[k]) : fc[k];
  }
  // class 4: pairs j < k, sign patterns ++, +-, -+, -- (the pairs on axis
  // k); the first axis j in a loop (its prefix picked from the unrolled
  // table), mid_jk grown by one term from (j, k - 1) to (j, k)
  for (int j = 0; j < D - 1; ++j) {
    float2 Lj = L3[0];
#pragma unroll
    for (int t = 1; t < D - 1; ++t)
      if (t == j) Lj = L3[t];
    float mid = 0.0f;
#pragma unroll
    for (int k = 1; k < D; ++k) {
      if (k > j) {
        if (k > j + 1) mid = (k > j + 2) ? op(mid, fc[k - 1]) : fc[k - 1];
        const float2 lm = (k > j + 1) ? op2(Lj, bc2(mid)) : Lj;
        const float2 sa = op2(bc2(lm.x), R3[k]);
        const float2 sb = op2(bc2(lm.y), R3[k]);
        bool zax = false, zay = false, zbx = false, zby = false;
        if constexpr (kFlag) {
          const bool zo = (zc & ~((1u << j) | (1u << k))) != 0u;
          const bool fjp = (z3 >> j) & 1u, fjm = (z3 >> (j + 16)) & 1u;
          const bool fkp = (z3 >> k) & 1u, fkm = (z3 >> (k + 16)) & 1u;
          zax = zo || fjp || fkp;
          zay = zo || fjp || fkm;
          zbx = zo || fjm || fkp;
          zby = zo || fjm || fkm;
        }
        const float2 va = g2z(sa, zax, zay);
        const float2 vb = g2z(sb, zbx, zby);
        S4.add(va.x);
        S4.add(va.y);
        S4.add(vb.x);
        S4.add(vb.y);
      }
    }
  }
  // class 5: the 2^D sign patterns m (bit j set: -lambda5 on axis j) in
  // ascending order, S = A[m_A] (+) (B_q (+) C_q), m = m_A + 2^LA q: A (the
  // chains over axes 0 .. LA-1) in registers, B_q and C_q (the chains over
  // the next LB axes and the rest, picked by the bits of q) formed once per
  // 2^LA patterns.  Patterns with even and odd m go to two accumulators.
  constexpr int LA = D < 4 ? D : 4;
  constexpr int LB = (D - LA) < 4 ? (D - LA) : 4;
  constexpr int NH = D - LA > 0 ? D - LA : 1;
  float A[1 << LA], p5h[NH], m5h[NH];
#pragma unroll
  for (int i = 0; i < LA; ++i) {
    const float xp = tab(kXP5, i), xm = tab(kXM5, i);
    const float fp = SF::phi(rp, i, xp), fm = SF::phi(rp, i, xm);
    if constexpr (kFlag)
      z5 |= ((unsigned)SF::flag(rp, i, xp) << i) | ((unsigned)SF::flag(rp, i, xm) << (i + 16));
    if (i == 0) {
      A[0] = kBase ? op(SF::base(rp), fp) : fp;
      A[1] = kBase ? op(SF::base(rp), fm) : fm;
    } else {
#pragma unroll
      for (int t = 0; t < (1 << i); ++t) {
        A[t + (1 << i)] = op(A[t], fm);
        A[t] = op(A[t], fp);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < D - LA; ++i) {
    const int j = LA + i;
    const float xp = tab(kXP5, j), xm = tab(kXM5, j);
    p5h[i] = SF::phi(rp, j, xp);
    m5h[i] = SF::phi(rp, j, xm);
    if constexpr (kFlag)
      z5 |= ((unsigned)SF::flag(rp, j, xp) << j) | ((unsigned)SF::flag(rp, j, xm) << (j + 16));
  }
  const unsigned dmask = (1u << D) - 1u;
  Acc<float> S5b;
  for (int q = 0; q < (1 << (D - LA)); ++q) {
    float bc = 0.0f;
    if constexpr (D > LA) {
      float bq = 0.0f, cq = 0.0f;
#pragma unroll
      for (int i = 0; i < D - LA; ++i) {
        const float t = ((q >> i) & 1) ? m5h[i] : p5h[i];
        if (i < LB)
          bq = i == 0 ? t : op(bq, t);
        else
          cq = i == LB ? t : op(cq, t);
      }
      bc = D - LA > LB ? op(bq, cq) : bq;
    }
#pragma unroll
    for (int lo = 0; lo < (1 << LA); lo += 2) {
      float2 S = make_float2(A[lo], A[lo + 1]);
      if constexpr (D > LA) S = op2(S, bc2(bc));
      bool zx = false, zy = false;
      if constexpr (kFlag) {
        const unsigned m = (unsigned)lo | ((unsigned)q << LA);
        zx = ((((~m) & z5) | (m & (z5 >> 16))) & dmask) != 0u;
        zy = ((((~(m + 1u)) & z5) | ((m + 1u) & (z5 >> 16))) & dmask) != 0u;
      }
      const float2 v = g2z(S, zx, zy);
      S5.add(v.x);
      S5b.add(v.y);
    }
  }
  o.s1 = S1.value();
  o.s2 = S2.value();
  o.s3 = S3.value();
  o.s4 = S4.value();
  o.s5 = __dadd_rn(S5.value(), S5b.value());
  o.dbest = dbest;
  o.kbest = kbest;
}

}  // namespace gmq
