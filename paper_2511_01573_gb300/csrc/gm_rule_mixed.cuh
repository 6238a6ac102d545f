// gm_rule_mixed.cuh -- mixed-precision rule-evaluation kernels (the f3
// form): the same rule, estimate and split axis as gm_rule.cuh's FP64
// kernel with the integrand in FP32.  Node coordinates are FP32, formed from
// the region's centre split into two FP32 parts (c = c_hi + c_lo) and its
// FP32 half-width; the integrand runs in FP32 and the class sums are FP32
// with TwoSum compensation; class sums, fourth differences, axis choice,
// rule values and error estimate are FP64 (region_finish64).
//   k_rule_mixed      any dimension, T = 1, 4 or 32 lanes per region (the
//                     lanes' compensated sums combined by a butterfly)
//   k_rule_mixed_reg  one thread per region, 3 <= d <= 12 known at compile
//                     time: the 2^d sign-pattern nodes walked in Gray-code
//                     order in registers (region_mixed_walk)
#pragma once

#include "gm_region32.cuh"
#include "gm_rule.cuh"

namespace gmq {

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
  const float l2 = (float)A.R.lam2, l3 = (float)A.R.lam3, l5 = (float)A.R.lam5;
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
    mixed_coord_rows(cv, hv, l2, l3, l5, xt + k * RB + q, d * RB);
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

// Mixed form, one thread per region, dimension D known at compile time:
// the sign-pattern nodes are walked in Gray-code order in registers
// (region_mixed_walk).
template <int FAM, int D>
__global__ void __launch_bounds__(kRuleBlock) k_rule_mixed_reg(const RuleArgs A) {
  static_assert(D >= 3 && D <= 16, "gray walk needs D >= 3");
  constexpr int RB = kRuleBlock;
  constexpr int d = D;
  // shared memory: the FP32 coordinate table and the FP32 parameters only
  // (the FP64 centres and half-widths the epilogue needs are read again
  // from the list), so more blocks fit on an SM
  extern __shared__ __align__(16) double smem[];
  float* xt = reinterpret_cast<float*>(smem);
  SmemParams<float>* P = reinterpret_cast<SmemParams<float>*>(xt + kXRows * d * RB);
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;
  for (int j = tid; j < d; j += RB) {
    P->a[j] = (float)A.P.a[j];
    P->u[j] = (float)A.P.u[j];
    P->b[j] = (float)A.P.b[j];
  }
  if (tid == 0) P->c0 = (float)A.P.c0;
  const float l2 = (float)A.R.lam2, l3 = (float)A.R.lam3, l5 = (float)A.R.lam5;
  for (int idx = tid; idx < d * RB; idx += RB) {
    const int k = idx / RB, q = idx - k * RB;
    const int64_t r = r0 + q;
    double cv = 0.5, hv = 0.25;
    if (r < A.n) {
      cv = A.c[(int64_t)k * A.ld + r];
      hv = A.h[(int64_t)k * A.ld + r];
    }
    mixed_coord_rows(cv, hv, l2, l3, l5, xt + k * RB + q, d * RB);
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
      [&](int k) { return A.c[(int64_t)k * A.ld + r]; },
      [&](int k) { return A.h[(int64_t)k * A.ld + r]; }, A.i7 + r, A.err + r,
      A.volfrac ? A.volfrac + r : nullptr, A.axis + r);
}

// Shared-memory bytes of k_rule_mixed_reg for dimension d.
inline size_t mixed_reg_smem_bytes(int d) {
  return ((size_t)sizeof(float) * kXRows * d * kRuleBlock + sizeof(SmemParams<float>) + 15) &
         ~(size_t)15;
}

template <int FAM, int D>
cudaError_t launch_mixed_reg_d(const RuleArgs& A, cudaStream_t s) {
  const size_t smem = mixed_reg_smem_bytes(D);
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


template <int FAM, int T>
cudaError_t launch_mixed_t(const RuleArgs& A, cudaStream_t s) {
  const int RB = kRuleBlock / T;
  const size_t smem = rule_smem_bytes(A.P.d, T, (int)sizeof(float));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rule_mixed<FAM, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (A.n + RB - 1) / RB;
  if (blocks == 0) return cudaSuccess;
  k_rule_mixed<FAM, T><<<(unsigned)blocks, kRuleBlock, smem, s>>>(A);
  return cudaGetLastError();
}

template <int FAM>
cudaError_t launch_mixed(int T, const RuleArgs& A, cudaStream_t s) {
  switch (T) {
    case 1: return launch_mixed_t<FAM, 1>(A, s);
    case 4: return launch_mixed_t<FAM, 4>(A, s);
    case 32: return launch_mixed_t<FAM, 32>(A, s);
    default: return cudaErrorInvalidValue;  // a block per region: FP64 only
  }
}

#define GMQ_DEFINE_RULE_FAMILY(FAMV)                                                   \
  template <>                                                                          \
  cudaError_t launch_rule_family<FAMV>(int precision, int T, const RuleArgs& A,         \
                                       cudaStream_t s) {                                \
    if (precision == GMQ_FP64) return launch_rule64<FAMV>(T, A, s);                    \
    if (precision == GMQ_MIXED && T == 1 && A.P.d >= 3 && A.P.d <= 12)                 \
      return launch_mixed_reg<FAMV>(A, s);                                             \
    if (precision == GMQ_MIXED) return launch_mixed<FAMV>(T, A, s);                    \
    return cudaErrorInvalidValue;                                                      \
  }

}  // namespace gmq
