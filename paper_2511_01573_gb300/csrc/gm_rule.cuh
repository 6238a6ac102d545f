// gm_rule.cuh -- rule-evaluation kernel (K1): the Genz-Malik degree-7 rule
// with its embedded degree-5 rule, the local error estimate and the
// fourth-difference split axis on every region of a sweep (paper Sec. 2).
//
// Mapping: a block of 128 threads owns RB = 128 / T consecutive regions, T
// threads ("lanes") per region, T in {1, 4, 32} (and 128, a block per
// region, in FP64).  The block
//   1. stages the regions' centres and half-widths from the structure-of-
//      arrays list into shared memory with coalesced loads (consecutive
//      threads read consecutive regions of one axis) and expands them into a
//      table of node coordinates c_k +- lambda h_k, one row per generator;
//   2. walks each class of nodes of each region by index: a node's axes and
//      signs are decoded from the bits of its index (centre; 4d axis nodes;
//      4 sign patterns per axis pair; the 2^d sign patterns of the last
//      class are the bits of the index itself), and its coordinates are read
//      from the table, so the only floating-point work per node is the
//      integrand and one accumulation;
//   3. combines the class sums over the T lanes with warp shuffles, finds the
//      split axis (argmax of the fourth differences) with a shuffle argmax,
//      and writes I7, |I7 - I5|, vol / vol(Omega) and the axis byte.
// FP64 (k_rule64): the per-region work is region_sums64 / region_finish64
// of gm_region64.cuh, whose fixed summation tree makes the results
// bit-identical for every T.  Mixed form (k_rule_mixed): node
// coordinates are formed in FP64 and rounded to FP32, the integrand runs in
// FP32 and the class sums are FP32 with TwoSum compensation, accumulated in
// node order per lane and combined over the lanes by a butterfly; class
// sums, fourth differences, axis choice, rule values and error estimate are
// FP64.  For one lane per region and 3 <= d <= 12 the mixed form walks the
// sign patterns in registers (k_rule_mixed_reg).
#pragma once

#include <type_traits>

#include "gm_region32.cuh"
#include "gm_region64.cuh"
#include "gmq_common.cuh"
#include "gmq_families.cuh"

namespace gmq {

// Shared-memory bytes of the rule kernel for dimension d, T lanes and an
// integrand type of `real_bytes` bytes.
inline size_t rule_smem_bytes(int d, int T, int real_bytes) {
  const int RB = kRuleBlock / T;
  size_t bytes = sizeof(double) * (size_t)2 * d * RB;          // centres, half-widths
  if (T > 1) bytes += sizeof(double) * ((size_t)4 * d * RB + RB);  // axis-node values, f(c)
  bytes += (size_t)real_bytes * kXRows * d * RB;                 // node coordinates
  bytes += sizeof(SmemParams<double>) + sizeof(unsigned short) * 128;
  return (bytes + 15) & ~(size_t)15;
}

// Mixed form, any dimension, T lanes per region.
template <int FAM, int T>
__global__ void __launch_bounds__(kRuleBlock) k_rule_mixed(const RuleArgs A) {
  using Real = float;
  constexpr int RB = kRuleBlock / T;
  extern __shared__ __align__(16) double smem[];
  const int d = A.P.d;
  double* cd = smem;                              // [d][RB] centres
  double* hd = cd + d * RB;                       // [d][RB] half-widths
  double* fv = hd + d * RB;                       // [4][d][RB] axis-node values (T > 1)
  double* f0s = fv + (T > 1 ? 4 * d * RB : 0);    // [RB] f(c)                   (T > 1)
  Real* xt = reinterpret_cast<Real*>(f0s + (T > 1 ? RB : 0));  // [kXRows][d][RB]
  SmemParams<Real>* P = reinterpret_cast<SmemParams<Real>*>(xt + kXRows * d * RB);
  unsigned short* pairs = reinterpret_cast<unsigned short*>(P + 1);

  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;

  // integrand parameters and the (j, k) pair table, j < k lexicographic
  for (int j = tid; j < d; j += kRuleBlock) {
    P->a[j] = (Real)A.P.a[j];
    P->u[j] = (Real)A.P.u[j];
    P->b[j] = (Real)A.P.b[j];
  }
  if (tid == 0) P->c0 = (Real)A.P.c0;
  const int npairs = d * (d - 1) / 2;
  for (int p = tid; p < npairs; p += kRuleBlock) {
    int j = 0, rem = p;
    while (rem >= d - 1 - j) {
      rem -= d - 1 - j;
      ++j;
    }
    pairs[p] = (unsigned short)((j << 8) | (j + 1 + rem));
  }

  // stage centres / half-widths and expand the node-coordinate table
  const double l2 = A.R.lam2, l3 = A.R.lam3, l5 = A.R.lam5;
  for (int idx = tid; idx < d * RB; idx += kRuleBlock) {
    const int k = idx / RB, q = idx - k * RB;
    const int64_t r = r0 + q;
    double cv = 0.5, hv = 0.25;
    if (r < A.n) {
      cv = A.c[(int64_t)k * A.ld + r];
      hv = A.h[(int64_t)k * A.ld + r];
    }
    cd[k * RB + q] = cv;
    hd[k * RB + q] = hv;
    xt[(kXC * d + k) * RB + q] = (Real)cv;
    xt[(kXP2 * d + k) * RB + q] = (Real)fma(l2, hv, cv);
    xt[(kXM2 * d + k) * RB + q] = (Real)fma(-l2, hv, cv);
    xt[(kXP3 * d + k) * RB + q] = (Real)fma(l3, hv, cv);
    xt[(kXM3 * d + k) * RB + q] = (Real)fma(-l3, hv, cv);
    xt[(kXP5 * d + k) * RB + q] = (Real)fma(l5, hv, cv);
    xt[(kXM5 * d + k) * RB + q] = (Real)fma(-l5, hv, cv);
  }
  __syncthreads();

  const int g = tid / T;     // region within the block
  const int lane = tid % T;  // lane within the region's group
  const int64_t r = r0 + g;
  const bool active = r < A.n;
  if constexpr (T == 1) {
    // one thread per region: the per-region work of the batched kernel
    if (!active) return;
    RegionSums o;
    region_mixed_flat<FAM>(
        *P, d, pairs, [&](int row, int j) -> float { return xt[(row * d + j) * RB + g]; },
        A.R.ratio, o);
    region_finish64(
        o, d, A.R.w7, A.R.w5, A.R.estimator ? A.R.nw : nullptr, A.R.vol_omega,
        [&](int k) { return cd[k * RB + g]; },
        [&](int k) { return hd[k * RB + g]; }, A.i7 + r, A.err + r,
        A.volfrac ? A.volfrac + r : nullptr, A.axis + r);
    return;
  }
  const int N = (int)A.R.nodes;
  const int b4 = 1 + 4 * d;             // first pair node
  const int b5 = b4 + 2 * d * (d - 1);  // first sign-class node
  const double ratio = A.R.ratio;

  Acc<Real> S1, S2, S3, S4, S5;
  double f0 = 0.0, q0 = 0.0, q1 = 0.0, q2 = 0.0, dbest = -1.0;
  int kbest = 0;

  if (active) {
    for (int i = lane; i < N; i += T) {
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
      auto X = [&](int j) -> Real {
        int row;
        if (kind == 5)
          row = ((m >> j) & 1u) ? kXM5 : kXP5;
        else
          row = (j == k1) ? r1 : ((j == k2) ? r2 : kXC);
        return xt[(row * d + j) * RB + g];
      };
      const Real v = Family<FAM>::template eval<Real>(*P, d, X);
      if (kind == 5) {
        S5.add(v);
      } else if (kind == 4) {
        S4.add(v);
      } else if (kind == 1) {
        S1.add(v);
        f0 = (double)v;
        if (T > 1) f0s[g] = (double)v;
      } else {
        if (kind == 2)
          S2.add(v);
        else
          S3.add(v);
        const double vd = (double)v;
        if (T == 1) {
          if (w == 0) {
            q0 = vd;
          } else if (w == 1) {
            q1 = vd;
          } else if (w == 2) {
            q2 = vd;
          } else {
            const double two_f0 = __dmul_rn(2.0, f0);
            const double t1 = __dsub_rn(__dadd_rn(q0, q1), two_f0);
            const double t2 = __dsub_rn(__dadd_rn(q2, vd), two_f0);
            const double D = fabs(__dsub_rn(t1, __dmul_rn(ratio, t2)));
            if (D > dbest) {
              dbest = D;
              kbest = k1;
            }
          }
        } else {
          fv[(w * d + k1) * RB + g] = vd;
        }
      }
    }
  }

  double s1 = S1.value(), s2 = S2.value(), s3 = S3.value(), s4 = S4.value(), s5 = S5.value();
  if (T > 1) {
    // class sums over the group's lanes
#pragma unroll
    for (int off = T / 2; off > 0; off >>= 1) {
      s1 += __shfl_xor_sync(0xffffffffu, s1, off, T);
      s2 += __shfl_xor_sync(0xffffffffu, s2, off, T);
      s3 += __shfl_xor_sync(0xffffffffu, s3, off, T);
      s4 += __shfl_xor_sync(0xffffffffu, s4, off, T);
      s5 += __shfl_xor_sync(0xffffffffu, s5, off, T);
    }
    __syncwarp();
    if (active) {
      f0 = f0s[g];
      for (int k = lane; k < d; k += T) {
        const double two_f0 = __dmul_rn(2.0, f0);
        const double t1 = __dsub_rn(__dadd_rn(fv[(0 * d + k) * RB + g], fv[(1 * d + k) * RB + g]), two_f0);
        const double t2 = __dsub_rn(__dadd_rn(fv[(2 * d + k) * RB + g], fv[(3 * d + k) * RB + g]), two_f0);
        const double D = fabs(__dsub_rn(t1, __dmul_rn(ratio, t2)));
        if (D > dbest) {
          dbest = D;
          kbest = k;
        }
      }
    }
    // argmax over lanes: larger D wins, lower axis on ties
#pragma unroll
    for (int off = T / 2; off > 0; off >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, dbest, off, T);
      const int ok = __shfl_xor_sync(0xffffffffu, kbest, off, T);
      if (od > dbest || (od == dbest && ok < kbest)) {
        dbest = od;
        kbest = ok;
      }
    }
  }

  if (active && lane == 0) {
    RegionSums o;
    o.s1 = s1;
    o.s2 = s2;
    o.s3 = s3;
    o.s4 = s4;
    o.s5 = s5;
    o.f0 = f0;
    o.dbest = dbest;
    o.kbest = kbest;
    region_finish64(
        o, d, A.R.w7, A.R.w5, A.R.estimator ? A.R.nw : nullptr, A.R.vol_omega,
        [&](int k) { return cd[k * RB + g]; },
        [&](int k) { return hd[k * RB + g]; }, A.i7 + r, A.err + r,
        A.volfrac ? A.volfrac + r : nullptr, A.axis + r);
  }
}

// FP64 rule kernel: same staging as k_rule_mixed, per-region work shared with the
// batched kernel (gm_region64.cuh).
template <int FAM, int T>
__global__ void __launch_bounds__(kRuleBlock) k_rule64(const RuleArgs A) {
  constexpr int RB = kRuleBlock / T;
  extern __shared__ __align__(16) double smem[];
  const int d = A.P.d;
  double* cd = smem;                                  // [d][RB] centres
  double* hd = cd + d * RB;                           // [d][RB] half-widths
  double* fv = hd + d * RB;                           // [4d + 1][RB] axis-node values, f(c)
  double* xt = fv + (T > 1 ? (4 * d + 1) * RB : 0);  // [kXRows][d][RB]
  SmemParams<double>* P = reinterpret_cast<SmemParams<double>*>(xt + kXRows * d * RB);
  unsigned short* pairs = reinterpret_cast<unsigned short*>(P + 1);

  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int j = tid; j < d; j += kRuleBlock) {
    P->a[j] = A.P.a[j];
    P->u[j] = A.P.u[j];
    P->b[j] = A.P.b[j];
  }
  if (tid == 0) P->c0 = A.P.c0;
  const int npairs = d * (d - 1) / 2;
  for (int p = tid; p < npairs; p += kRuleBlock) {
    int j = 0, rem = p;
    while (rem >= d - 1 - j) {
      rem -= d - 1 - j;
      ++j;
    }
    pairs[p] = (unsigned short)((j << 8) | (j + 1 + rem));
  }
  const double l2 = A.R.lam2, l3 = A.R.lam3, l5 = A.R.lam5;
  for (int idx = tid; idx < d * RB; idx += kRuleBlock) {
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
  __syncthreads();

  const int g = tid / T;
  const int64_t r = r0 + g;
  if (r >= A.n) return;  // the whole group: its lanes share the region
  auto tab = [&](int row, int j) -> double { return xt[(row * d + j) * RB + g]; };
  RegionSums o;
  region_sums64<FAM, T>(*P, d, pairs, tab, fv + g, RB, A.R.ratio, o);
  if ((tid & (T - 1)) == 0)
    region_finish64(
        o, d, A.R.w7, A.R.w5, A.R.estimator ? A.R.nw : nullptr, A.R.vol_omega,
        [&](int k) { return cd[k * RB + g]; },
        [&](int k) { return hd[k * RB + g]; }, A.i7 + r, A.err + r,
        A.volfrac ? A.volfrac + r : nullptr, A.axis + r);
}

// Mixed form, one thread per region, dimension D known at compile time:
// the sign-pattern nodes are walked in Gray-code order in registers
// (region_mixed_walk).
template <int FAM, int D>
__global__ void __launch_bounds__(kRuleBlock) k_rule_mixed_reg(const RuleArgs A) {
  static_assert(D >= 3 && D <= 16, "gray walk needs D >= 3");
  constexpr int RB = kRuleBlock;
  constexpr int d = D;
  extern __shared__ __align__(16) double smem[];
  double* cd = smem;
  double* hd = cd + d * RB;
  float* xt = reinterpret_cast<float*>(hd + d * RB);
  SmemParams<float>* P = reinterpret_cast<SmemParams<float>*>(xt + kXRows * d * RB);
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int j = tid; j < d; j += RB) {
    P->a[j] = (float)A.P.a[j];
    P->u[j] = (float)A.P.u[j];
    P->b[j] = (float)A.P.b[j];
  }
  if (tid == 0) P->c0 = (float)A.P.c0;
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
    xt[(kXC * d + k) * RB + q] = (float)cv;
    xt[(kXP2 * d + k) * RB + q] = (float)fma(l2, hv, cv);
    xt[(kXM2 * d + k) * RB + q] = (float)fma(-l2, hv, cv);
    xt[(kXP3 * d + k) * RB + q] = (float)fma(l3, hv, cv);
    xt[(kXM3 * d + k) * RB + q] = (float)fma(-l3, hv, cv);
    xt[(kXP5 * d + k) * RB + q] = (float)fma(l5, hv, cv);
    xt[(kXM5 * d + k) * RB + q] = (float)fma(-l5, hv, cv);
  }
  __syncthreads();
  const int g = tid;
  const int64_t r = r0 + g;
  if (r >= A.n) return;
  RegionSums o;
  region_mixed_walk<FAM, D>(
      *P, [&](int row, int j) -> float { return xt[(row * d + j) * RB + g]; }, A.R.ratio, o);
  region_finish64(
      o, d, A.R.w7, A.R.w5, A.R.estimator ? A.R.nw : nullptr, A.R.vol_omega,
      [&](int k) { return cd[k * RB + g]; },
      [&](int k) { return hd[k * RB + g]; }, A.i7 + r, A.err + r,
      A.volfrac ? A.volfrac + r : nullptr, A.axis + r);
}

template <int FAM, int D>
cudaError_t launch_mixed_reg_d(const RuleArgs& A, cudaStream_t s) {
  const size_t smem = rule_smem_bytes(D, 1, (int)sizeof(float));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rule_mixed_reg<FAM, D>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (A.n + kRuleBlock - 1) / kRuleBlock;
  if (blocks == 0) return cudaSuccess;
  k_rule_mixed_reg<FAM, D><<<(unsigned)blocks, kRuleBlock, smem, s>>>(A);
  return cudaGetLastError();
}

// The register-walk variant exists for 3 <= d <= 12; returns
// cudaErrorNotSupported for other d.
template <int FAM>
cudaError_t launch_mixed_reg(const RuleArgs& A, cudaStream_t s) {
  switch (A.P.d) {
    case 3: return launch_mixed_reg_d<FAM, 3>(A, s);
    case 4: return launch_mixed_reg_d<FAM, 4>(A, s);
    case 5: return launch_mixed_reg_d<FAM, 5>(A, s);
    case 6: return launch_mixed_reg_d<FAM, 6>(A, s);
    case 7: return launch_mixed_reg_d<FAM, 7>(A, s);
    case 8: return launch_mixed_reg_d<FAM, 8>(A, s);
    case 9: return launch_mixed_reg_d<FAM, 9>(A, s);
    case 10: return launch_mixed_reg_d<FAM, 10>(A, s);
    case 11: return launch_mixed_reg_d<FAM, 11>(A, s);
    case 12: return launch_mixed_reg_d<FAM, 12>(A, s);
    default: return cudaErrorNotSupported;
  }
}

// Launch the rule kernel of one family for T lanes per region.
template <int FAM>
cudaError_t launch_rule_family(int precision, int T, const RuleArgs& A, cudaStream_t s);

template <int FAM, int T, class Real>
cudaError_t launch_rule_t(const RuleArgs& A, cudaStream_t s) {
  const int RB = kRuleBlock / T;
  const size_t smem = rule_smem_bytes(A.P.d, T, (int)sizeof(Real));
  void (*kern)(const RuleArgs);
  if constexpr (std::is_same<Real, double>::value)
    kern = k_rule64<FAM, T>;
  else
    kern = k_rule_mixed<FAM, T>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (A.n + RB - 1) / RB;
  if (blocks == 0) return cudaSuccess;
  kern<<<(unsigned)blocks, kRuleBlock, smem, s>>>(A);
  return cudaGetLastError();
}

template <int FAM, class Real>
cudaError_t launch_rule_real(int T, const RuleArgs& A, cudaStream_t s) {
  switch (T) {
    case 1: return launch_rule_t<FAM, 1, Real>(A, s);
    case 4: return launch_rule_t<FAM, 4, Real>(A, s);
    case 32: return launch_rule_t<FAM, 32, Real>(A, s);
    case 128:  // a block per region: FP64 only
      if constexpr (std::is_same<Real, double>::value) return launch_rule_t<FAM, 128, Real>(A, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

#define GMQ_DEFINE_RULE_FAMILY(FAMV)                                                   \
  template <>                                                                          \
  cudaError_t launch_rule_family<FAMV>(int precision, int T, const RuleArgs& A,         \
                                       cudaStream_t s) {                                \
    if (precision == GMQ_FP64) return launch_rule_real<FAMV, double>(T, A, s);         \
    if (precision == GMQ_MIXED && T == 1 && A.P.d >= 3 && A.P.d <= 12)                 \
      return launch_mixed_reg<FAMV>(A, s);                                             \
    if (precision == GMQ_MIXED) return launch_rule_real<FAMV, float>(T, A, s);         \
    return cudaErrorInvalidValue;                                                      \
  }

}  // namespace gmq
