// gm_rule.cuh -- rule-evaluation kernel (K1): the Genz-Malik degree-7 rule
// with its embedded degree-5 rule, the local error estimate and the
// fourth-difference split axis on every region of a sweep (paper Sec. 2).
//
// Mapping: a block of 128 threads owns RB = 128 / T consecutive regions, T
// threads ("lanes") per region, T in {1, 4, 32}.  The block
//   1. stages the regions' centres and half-widths from the structure-of-
//      arrays list into shared memory with coalesced loads (consecutive
//      threads read consecutive regions of one axis) and expands them into a
//      table of node coordinates c_k +- lambda h_k, one row per generator;
//   2. walks the flat node index i = 0 .. N(d)-1 of each region, lane l of a
//      region taking i = l, l+T, ...; a node's class, axes and signs are
//      decoded from the bits of i (centre; 4d axis nodes; 4 sign patterns
//      per axis pair; the 2^d sign patterns of the last class are the bits
//      of i itself), and its coordinates are read from the table, so the
//      only FP64 work per node is the integrand and one accumulation;
//   3. reduces the five class sums over the T lanes with warp shuffles,
//      finds the split axis (argmax of the fourth differences) with a
//      shuffle argmax, and writes I7, |I7 - I5|, vol / vol(Omega) and the
//      axis byte.
// With T = 1 the class sums are accumulated in the same node order as the
// plain definition (centre; per axis +l2, -l2, +l3, -l3; pairs j < k with
// sign patterns ++, +-, -+, --; sign patterns m = 0 .. 2^d - 1).
#pragma once

#include "gmq_common.cuh"
#include "gmq_families.cuh"

namespace gmq {

// Shared-memory bytes of the rule kernel for dimension d and T lanes.
inline size_t rule_smem_bytes(int d, int T) {
  const int RB = kRuleBlock / T;
  size_t dbl = (size_t)kRows * d * RB;
  if (T > 1) dbl += (size_t)4 * d * RB + RB;
  size_t bytes = dbl * sizeof(double) + sizeof(SmemParams) + sizeof(unsigned short) * 128;
  return (bytes + 15) & ~(size_t)15;
}

template <int FAM, int T>
__global__ void __launch_bounds__(kRuleBlock) k_rule_f64(const RuleArgs A) {
  constexpr int RB = kRuleBlock / T;
  extern __shared__ __align__(16) double smem[];
  const int d = A.P.d;
  double* tab = smem;  // [kRows][d][RB]
  double* fv = tab + kRows * d * RB;            // [4][d][RB]   (T > 1)
  double* f0s = fv + (T > 1 ? 4 * d * RB : 0);  // [RB]         (T > 1)
  SmemParams* P = reinterpret_cast<SmemParams*>(f0s + (T > 1 ? RB : 0));
  unsigned short* pairs = reinterpret_cast<unsigned short*>(P + 1);

  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RB;

  // integrand parameters and the (j, k) pair table, j < k lexicographic
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
    tab[(kC * d + k) * RB + q] = cv;
    tab[(kH * d + k) * RB + q] = hv;
    tab[(kP2 * d + k) * RB + q] = fma(l2, hv, cv);
    tab[(kM2 * d + k) * RB + q] = fma(-l2, hv, cv);
    tab[(kP3 * d + k) * RB + q] = fma(l3, hv, cv);
    tab[(kM3 * d + k) * RB + q] = fma(-l3, hv, cv);
    tab[(kP5 * d + k) * RB + q] = fma(l5, hv, cv);
    tab[(kM5 * d + k) * RB + q] = fma(-l5, hv, cv);
  }
  __syncthreads();

  const int g = tid / T;     // region within the block
  const int lane = tid % T;  // lane within the region's group
  const int64_t r = r0 + g;
  const bool active = r < A.n;
  const int N = (int)A.R.nodes;
  const int b4 = 1 + 4 * d;               // first pair node
  const int b5 = b4 + 2 * d * (d - 1);    // first sign-class node
  const double ratio = A.R.ratio;

  double S1 = 0.0, S2 = 0.0, S3 = 0.0, S4 = 0.0, S5 = 0.0;
  double f0 = 0.0, q0 = 0.0, q1 = 0.0, q2 = 0.0, dbest = -1.0;
  int kbest = 0;

  if (active) {
    for (int i = lane; i < N; i += T) {
      int kind, k1 = -1, r1 = kC, k2 = -1, r2 = kC, w = 0;
      unsigned m = 0u;
      if (i == 0) {
        kind = 1;
      } else if (i < b4) {
        const int q = i - 1;
        k1 = q >> 2;
        w = q & 3;
        r1 = kP2 + w;
        kind = (w < 2) ? 2 : 3;
      } else if (i < b5) {
        const int q = i - b4;
        const unsigned pr = pairs[q >> 2];
        k1 = (int)(pr >> 8);
        k2 = (int)(pr & 255u);
        r1 = (q & 2) ? kM3 : kP3;
        r2 = (q & 1) ? kM3 : kP3;
        kind = 4;
      } else {
        m = (unsigned)(i - b5);
        kind = 5;
      }
      auto X = [&](int j) -> double {
        int row;
        if (kind == 5)
          row = ((m >> j) & 1u) ? kM5 : kP5;
        else
          row = (j == k1) ? r1 : ((j == k2) ? r2 : kC);
        return tab[(row * d + j) * RB + g];
      };
      const double v = Family<FAM>::eval(*P, d, X);
      if (kind == 5) {
        S5 += v;
      } else if (kind == 4) {
        S4 += v;
      } else if (kind == 1) {
        S1 += v;
        f0 = v;
        if (T > 1) f0s[g] = v;
      } else {
        if (kind == 2)
          S2 += v;
        else
          S3 += v;
        if (T == 1) {
          if (w == 0) {
            q0 = v;
          } else if (w == 1) {
            q1 = v;
          } else if (w == 2) {
            q2 = v;
          } else {
            const double two_f0 = __dmul_rn(2.0, f0);
            const double t1 = __dsub_rn(__dadd_rn(q0, q1), two_f0);
            const double t2 = __dsub_rn(__dadd_rn(q2, v), two_f0);
            const double D = fabs(__dsub_rn(t1, __dmul_rn(ratio, t2)));
            if (D > dbest) {
              dbest = D;
              kbest = k1;
            }
          }
        } else {
          fv[(w * d + k1) * RB + g] = v;
        }
      }
    }
  }

  if (T > 1) {
    // class sums over the group's lanes
#pragma unroll
    for (int off = T / 2; off > 0; off >>= 1) {
      S1 += __shfl_xor_sync(0xffffffffu, S1, off, T);
      S2 += __shfl_xor_sync(0xffffffffu, S2, off, T);
      S3 += __shfl_xor_sync(0xffffffffu, S3, off, T);
      S4 += __shfl_xor_sync(0xffffffffu, S4, off, T);
      S5 += __shfl_xor_sync(0xffffffffu, S5, off, T);
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
    // volume, rule values and error estimate
    double vol = 1.0;
    for (int k = 0; k < d; ++k) vol = __dmul_rn(vol, __dmul_rn(2.0, tab[(kH * d + k) * RB + g]));
    const double* w7 = A.R.w7;
    const double* w5 = A.R.w5;
    double s7 = __dmul_rn(w7[0], S1);
    s7 = __dadd_rn(s7, __dmul_rn(w7[1], S2));
    s7 = __dadd_rn(s7, __dmul_rn(w7[2], S3));
    s7 = __dadd_rn(s7, __dmul_rn(w7[3], S4));
    s7 = __dadd_rn(s7, __dmul_rn(w7[4], S5));
    double s5 = __dmul_rn(w5[0], S1);
    s5 = __dadd_rn(s5, __dmul_rn(w5[1], S2));
    s5 = __dadd_rn(s5, __dmul_rn(w5[2], S3));
    s5 = __dadd_rn(s5, __dmul_rn(w5[3], S4));
    const double i7 = __dmul_rn(vol, s7);
    const double i5 = __dmul_rn(vol, s5);
    // split axis: flat differences -> widest axis (lowest index on ties)
    const double flat_thr = __dadd_rn(__dmul_rn(1e-14, fabs(f0)), 1e-300);
    int ax = kbest;
    if (!(dbest > flat_thr)) {
      ax = 0;
      double hb = tab[(kH * d + 0) * RB + g];
      for (int k = 1; k < d; ++k) {
        const double hk = tab[(kH * d + k) * RB + g];
        if (hk > hb) {
          hb = hk;
          ax = k;
        }
      }
    }
    // round-off guard: bisection along ax must move the centre
    const double cs = tab[(kC * d + ax) * RB + g];
    const double hh = __dmul_rn(0.5, tab[(kH * d + ax) * RB + g]);
    const bool bad = (hh == 0.0) || (__dsub_rn(cs, hh) == cs) || (__dadd_rn(cs, hh) == cs);
    A.i7[r] = i7;
    A.err[r] = fabs(__dsub_rn(i7, i5));
    if (A.volfrac) A.volfrac[r] = __ddiv_rn(vol, A.R.vol_omega);
    A.axis[r] = (uint8_t)(ax | (bad ? 0x80 : 0));
  }
}

// Launch the rule kernel of one family for T lanes per region.
template <int FAM>
cudaError_t launch_rule_family(int precision, int T, const RuleArgs& A, cudaStream_t s);

template <int FAM, int T>
cudaError_t launch_rule_t(const RuleArgs& A, cudaStream_t s) {
  const int RB = kRuleBlock / T;
  const size_t smem = rule_smem_bytes(A.P.d, T);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rule_f64<FAM, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (A.n + RB - 1) / RB;
  if (blocks == 0) return cudaSuccess;
  k_rule_f64<FAM, T><<<(unsigned)blocks, kRuleBlock, smem, s>>>(A);
  return cudaGetLastError();
}

#define GMQ_DEFINE_RULE_FAMILY(FAMV)                                                   \
  template <>                                                                          \
  cudaError_t launch_rule_family<FAMV>(int precision, int T, const RuleArgs& A,         \
                                       cudaStream_t s) {                                \
    if (precision != GMQ_FP64) return cudaErrorNotSupported;                          \
    switch (T) {                                                                       \
      case 1: return launch_rule_t<FAMV, 1>(A, s);                                     \
      case 4: return launch_rule_t<FAMV, 4>(A, s);                                     \
      case 32: return launch_rule_t<FAMV, 32>(A, s);                                   \
      default: return cudaErrorInvalidValue;                                           \
    }                                                                                  \
  }

}  // namespace gmq
