// gm_rule.cuh -- FP64 rule-evaluation kernel (K1): the Genz-Malik degree-7
// rule with its embedded degree-5 rule, the local error estimate and the
// fourth-difference split axis on every region of a sweep (paper Sec. 2).
// The mixed-precision kernels are in gm_rule_mixed.cuh.
//
// Mapping: a block of 128 threads owns RB = 128 / T consecutive regions, T
// threads ("lanes") per region, T in {1, 4, 32, 128} (128: a block per
// region).  Each group
//   1. reads its region's centres and half-widths from the structure-of-
//      arrays list (consecutive threads read consecutive regions of one
//      axis: coalesced) and builds the region's separable workspace in
//      shared memory: the integrand's per-axis terms at the seven
//      coordinate values of each axis, their prefix and suffix chains and
//      the class-5 partial chains (gm_region64.cuh);
//   2. walks each class of nodes by index: a node's axes and signs are
//      decoded from the bits of its index (centre; 4d axis nodes; 4 sign
//      patterns per axis pair; the 2^d sign patterns of the last class are
//      the bits of the index itself), its S combined from the workspace in
//      one or two operations, so the FP64 work per node is the integrand's
//      outer function and one accumulation;
//   3. combines the class sums over the T lanes, finds the split axis
//      (argmax of the fourth differences) and writes I7, the error estimate,
//      vol / vol(Omega) and the axis byte.
// The per-region work is region_sums64 / region_finish64 of gm_region64.cuh,
// whose fixed summation tree makes the results bit-identical for every T.
#pragma once

#include "gm_region64.cuh"
#include "gmq_common.cuh"
#include "gmq_families.cuh"

namespace gmq {

// Shared-memory bytes of the mixed rule kernels and the node-wise FP64
// kernel for dimension d, T lanes and an integrand type of `real_bytes`
// bytes.
inline size_t rule_smem_bytes(int d, int T, int real_bytes) {
  const int RB = kRuleBlock / T;
  size_t bytes = sizeof(double) * (size_t)2 * d * RB;          // centres, half-widths
  if (T > 1) bytes += sizeof(double) * ((size_t)4 * d * RB + RB);  // axis-node values, f(c)
  bytes += (size_t)real_bytes * kXRows * d * RB;                 // node coordinates
  bytes += sizeof(SmemParams<double>) + sizeof(unsigned short) * 128;
  return (bytes + 15) & ~(size_t)15;
}

// Shared-memory bytes of the FP64 rule kernel: RB workspaces of the region
// layout, the family parameters and the pair table.
inline size_t rule64_smem_bytes(int d, int T, bool flag) {
  const int RB = kRuleBlock / T;
  size_t bytes = sizeof(double) * (size_t)sep_layout(d, flag, T > 1).words * RB;
  bytes += sizeof(SmemParams<double>) + sizeof(unsigned short) * 128;
  return (bytes + 15) & ~(size_t)15;
}

// FP64 rule kernel; per-region work shared with the batched kernel
// (gm_region64.cuh).
template <int FAM, int T>
__global__ void __launch_bounds__(kRuleBlock) k_rule64(const RuleArgs A) {
  constexpr int RB = kRuleBlock / T;
  extern __shared__ __align__(16) double smem[];
  const int d = A.P.d;
  const int words = sep_layout(d, Sep<FAM>::kFlag, T > 1).words;
  double* wsp = smem;  // [words][RB] region workspaces
  SmemParams<double>* P = reinterpret_cast<SmemParams<double>*>(wsp + (size_t)words * RB);
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
  __syncthreads();

  const int g = tid / T;
  const int64_t r = r0 + g;
  if (r >= A.n) return;  // the whole group: its lanes share the region
  const double* C = A.c + r;
  const double* H = A.h + r;
  const int64_t ld = A.ld;
  auto ch = [&](int k, double& c, double& h) {
    c = C[(int64_t)k * ld];
    h = H[(int64_t)k * ld];
  };
  RegionSums o;
  region_sums64<FAM, T>(*P, d, pairs, ch, A.R.lam2, A.R.lam3, A.R.lam5, wsp + g, RB, A.R.ratio,
                        o);
  if ((tid & (T - 1)) == 0)
    region_finish64(
        o, d, A.R.w7, A.R.w5, A.R.estimator ? A.R.nw : nullptr, A.R.vol_omega,
        [&](int k) { return C[(int64_t)k * ld]; }, [&](int k) { return H[(int64_t)k * ld]; },
        A.i7 + r, A.err + r, A.volfrac ? A.volfrac + r : nullptr, A.axis + r);
}


// FP64 rule kernel with node-wise evaluation (GMQ_EVAL_NODEWISE): the
// block stages its regions' centres and half-widths and a table of the
// node coordinates c_k +- lambda h_k in shared memory (the mixed kernels'
// layout, rule_smem_bytes), and every node evaluates f from its
// coordinates.
template <int FAM, int T>
__global__ void __launch_bounds__(kRuleBlock) k_rule64_nodewise(const RuleArgs A) {
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
  region_sums64_nodewise<FAM, T>(*P, d, pairs, tab, fv + g, RB, A.R.ratio, o);
  if ((tid & (T - 1)) == 0)
    region_finish64(
        o, d, A.R.w7, A.R.w5, A.R.estimator ? A.R.nw : nullptr, A.R.vol_omega,
        [&](int k) { return cd[k * RB + g]; },
        [&](int k) { return hd[k * RB + g]; }, A.i7 + r, A.err + r,
        A.volfrac ? A.volfrac + r : nullptr, A.axis + r);
}


// Launch the rule kernel of one family (precision, T lanes per region);
// defined per family by GMQ_DEFINE_RULE_FAMILY (gm_rule_mixed.cuh).
template <int FAM>
cudaError_t launch_rule_family(int precision, int T, const RuleArgs& A, cudaStream_t s);

template <int FAM, int T>
cudaError_t launch_rule64_t(const RuleArgs& A, cudaStream_t s) {
  const int RB = kRuleBlock / T;
  if (A.nodewise) {
    const size_t smem = rule_smem_bytes(A.P.d, T, (int)sizeof(double));
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_rule64_nodewise<FAM, T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (A.n + RB - 1) / RB;
    if (blocks == 0) return cudaSuccess;
    k_rule64_nodewise<FAM, T><<<(unsigned)blocks, kRuleBlock, smem, s>>>(A);
    return cudaGetLastError();
  }
  const size_t smem = rule64_smem_bytes(A.P.d, T, Sep<FAM>::kFlag);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rule64<FAM, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (A.n + RB - 1) / RB;
  if (blocks == 0) return cudaSuccess;
  k_rule64<FAM, T><<<(unsigned)blocks, kRuleBlock, smem, s>>>(A);
  return cudaGetLastError();
}

template <int FAM>
cudaError_t launch_rule64(int T, const RuleArgs& A, cudaStream_t s) {
  switch (T) {
    case 1: return launch_rule64_t<FAM, 1>(A, s);
    case 4: return launch_rule64_t<FAM, 4>(A, s);
    case 32: return launch_rule64_t<FAM, 32>(A, s);
    case 128: return launch_rule64_t<FAM, 128>(A, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gmq
