// gm_gk.cuh -- the tensor-product Gauss-Kronrod (7, 15) rule (paper Sec. 3
// names a tensor-product Gauss-Kronrod rule as one of the rules the method
// can use, without its order or split axis -- the readings here are the
// classic G7/K15 pair and the directional error estimates).
//
// On a region c +- h the rule evaluates f at the 15^d nodes c + h o xi,
// xi in {K15 nodes}^d, and forms
//   I_K = prod h_k sum_i (prod_k wK[i_k]) f,   I_G likewise with the G7
//   weights (0 at the 8 Kronrod-only nodes),   eps = |I_K - I_G|,
//   E_k = prod h_k |sum_i (prod_{j != k} wK[i_j]) (wK[i_k] - wG[i_k]) f|,
// the error estimate in direction k; the split axis is argmax_k E_k (lowest
// index on ties), or the widest axis when every E_k is below 1e-11 of the
// magnitude of the terms (prod h_k sum |wK f|).  d <= GMQ_GK_MAX_DIM.
//
// Mapping: one warp per region, four regions per 128-thread block.  The
// node grid is walked by rows -- a row fixes the digits of axes 1..d-1 and
// runs axis 0 over its 15 nodes -- lane l taking rows l, l + 32, ...; the
// weight products of axes >= 1 and the E_k terms of axes >= 1 are formed
// once per row (E_k += r_k[i_k] * (row sum of wK f), r = 1 - wG / wK), so
// per node the FP64 work is the integrand and five operations.  Warp
// butterflies combine the lanes' sums in a fixed order.
#pragma once

#include "gmq_common.cuh"
#include "gmq_families.cuh"

namespace gmq {

// 1-D tables on [-1, 1], ascending nodes; wg = 0 at Kronrod-only nodes;
// r = 1 - wg / wk.
struct GkConst {
  double x[15], wk[15], wg[15], r[15];
};

// Computed once on the host (gmq_api.cu); each context keeps a device copy.
const GkConst& gk_const();

struct GkArgs {
  RuleArgs A;
  const GkConst* K;  // device copy of the tables
};

constexpr int kGkWarps = 4;  // regions per block

template <int FAM>
__global__ void __launch_bounds__(32 * kGkWarps) k_rule_gk(const GkArgs G) {
  __shared__ GkConst K;
  __shared__ SmemParams<double> P;
  __shared__ double xt[kGkWarps][GMQ_GK_MAX_DIM * 15];  // node coordinates per axis
  __shared__ double xs[kGkWarps][GMQ_GK_MAX_DIM][32];   // each lane's current node
  const RuleArgs& A = G.A;
  const int d = A.P.d;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 60; i += blockDim.x) (&K.x[0])[i] = (&G.K->x[0])[i];
  for (int j = tid; j < d; j += blockDim.x) {
    P.a[j] = A.P.a[j];
    P.u[j] = A.P.u[j];
    P.b[j] = A.P.b[j];
  }
  if (tid == 0) P.c0 = A.P.c0;
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * kGkWarps + w;
  const bool active = r < A.n;
  if (active)
    for (int q = lane; q < d * 15; q += 32) {
      const int k = q / 15, j = q - 15 * k;
      xt[w][q] = fma(K.x[j], A.h[(int64_t)k * A.ld + r], A.c[(int64_t)k * A.ld + r]);
    }
  __syncthreads();
  if (!active) return;  // the whole warp: its lanes share the region
  int rows = 1;
  for (int k = 1; k < d; ++k) rows *= 15;
  double SK = 0.0, SG = 0.0, SA = 0.0;
  double E[GMQ_GK_MAX_DIM];
#pragma unroll
  for (int k = 0; k < GMQ_GK_MAX_DIM; ++k) E[k] = 0.0;
  auto X = [&](int j) -> double { return xs[w][j][lane]; };
  for (int row = lane; row < rows; row += 32) {
    // digits of axes 1..d-1, their weight products and coordinates
    int q = row;
    double wr = 1.0, gr = 1.0;
    int dig[GMQ_GK_MAX_DIM];
#pragma unroll
    for (int k = 1; k < GMQ_GK_MAX_DIM; ++k) {
      if (k < d) {
        dig[k] = q % 15;
        q /= 15;
        wr = wr * K.wk[dig[k]];
        gr = gr * K.wg[dig[k]];
        xs[w][k][lane] = xt[w][k * 15 + dig[k]];
      }
    }
    double rk = 0.0, rg = 0.0, ra = 0.0, e0 = 0.0;
    for (int j = 0; j < 15; ++j) {
      xs[w][0][lane] = xt[w][j];
      const double v = Family<FAM>::template eval<double>(P, d, X);
      const double t = __dmul_rn(__dmul_rn(K.wk[j], wr), v);  // wK-product * f
      rk = __dadd_rn(rk, t);
      rg = fma(__dmul_rn(K.wg[j], gr), v, rg);
      ra = fma(__dmul_rn(K.wk[j], wr), fabs(v), ra);
      e0 = fma(K.r[j], t, e0);
    }
    SK = __dadd_rn(SK, rk);
    SG = __dadd_rn(SG, rg);
    SA = __dadd_rn(SA, ra);
    E[0] = __dadd_rn(E[0], e0);
#pragma unroll
    for (int k = 1; k < GMQ_GK_MAX_DIM; ++k)
      if (k < d) E[k] = fma(K.r[dig[k]], rk, E[k]);
  }
  // combine the lanes (fixed butterfly order)
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    SK += __shfl_xor_sync(0xffffffffu, SK, off);
    SG += __shfl_xor_sync(0xffffffffu, SG, off);
    SA += __shfl_xor_sync(0xffffffffu, SA, off);
#pragma unroll
    for (int k = 0; k < GMQ_GK_MAX_DIM; ++k) E[k] += __shfl_xor_sync(0xffffffffu, E[k], off);
  }
  if (lane != 0) return;
  double hprod = 1.0, vol = 1.0;
  for (int k = 0; k < d; ++k) {
    const double hk = A.h[(int64_t)k * A.ld + r];
    hprod = __dmul_rn(hprod, hk);
    vol = __dmul_rn(vol, __dmul_rn(2.0, hk));
  }
  const double ik = __dmul_rn(hprod, SK), ig = __dmul_rn(hprod, SG);
  const double scale = __dmul_rn(hprod, SA);
  int best = 0;
  double eb = __dmul_rn(hprod, fabs(E[0]));
#pragma unroll
  for (int k = 1; k < GMQ_GK_MAX_DIM; ++k) {
    if (k < d) {
      const double ek = __dmul_rn(hprod, fabs(E[k]));
      if (ek > eb) {
        eb = ek;
        best = k;
      }
    }
  }
  int ax = best;
  if (!(eb > __dadd_rn(__dmul_rn(1e-11, scale), 1e-300))) {
    ax = 0;
    double hb = A.h[r];
    for (int k = 1; k < d; ++k) {
      const double hk = A.h[(int64_t)k * A.ld + r];
      if (hk > hb) {
        hb = hk;
        ax = k;
      }
    }
  }
  const double cs = A.c[(int64_t)ax * A.ld + r];
  const double hh = __dmul_rn(0.5, A.h[(int64_t)ax * A.ld + r]);
  const bool bad = (hh == 0.0) || (__dsub_rn(cs, hh) == cs) || (__dadd_rn(cs, hh) == cs);
  A.i7[r] = ik;
  A.err[r] = fabs(__dsub_rn(ik, ig));
  if (A.volfrac) A.volfrac[r] = __ddiv_rn(vol, A.R.vol_omega);
  A.axis[r] = (uint8_t)(ax | (bad ? 0x80 : 0));
}

template <int FAM>
cudaError_t launch_rule_gk_family(const GkArgs& G, cudaStream_t s) {
  const int64_t blocks = (G.A.n + kGkWarps - 1) / kGkWarps;
  if (blocks == 0) return cudaSuccess;
  k_rule_gk<FAM><<<(unsigned)blocks, 32 * kGkWarps, 0, s>>>(G);
  return cudaGetLastError();
}

#define GMQ_DEFINE_GK_FAMILY(FAMV) \
  template cudaError_t launch_rule_gk_family<FAMV>(const GkArgs& G, cudaStream_t s);

}  // namespace gmq
