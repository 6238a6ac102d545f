// gm_batch_mixed.cuh -- rule evaluation of the batched form in the mixed
// precision, one kernel per integrand family (instantiated with the other
// per-family kernels in gm_rule_inst.cu).  The batch is in family order, so
// each family's regions are one contiguous range of the list; a launch walks
// its family's range on a persistent grid, one thread per region, with the
// single-integral mixed path's
// per-region code (gm_region32.cuh): the Gray-code register walk for
// 3 <= d <= 12, the generic one-thread form otherwise.  So every region gets
// the bits gmq_integrate's mixed path with one lane per region gives it.
#pragma once

#include "gm_batch.cuh"
#include "gm_region32.cuh"

namespace gmq {

// Shared memory of the batched mixed rule kernel: per thread the region's
// FP32 coordinate table, then the pair tables of every dimension 2 .. dmax
// (the FP64 centres and half-widths the epilogue needs are read again from
// the list).
inline size_t batch_rule_mixed_smem(int dmax) {
  size_t bytes = sizeof(float) * (size_t)kXRows * dmax * kBatchRuleBlock;
  bytes += sizeof(unsigned short) * (size_t)(dmax + 1) * dmax * (dmax - 1) / 6;
  return (bytes + 15) & ~(size_t)15;
}

template <int FAM>
__global__ void __launch_bounds__(kBatchRuleBlock) k_batch_rule_mixed(const BatchArgs B) {
  constexpr int RB = kBatchRuleBlock;
  extern __shared__ __align__(16) double smem[];
  const int dm = B.dmax;
  float* xt = reinterpret_cast<float*>(smem);  // [kXRows][dm][RB]
  unsigned short* pairs_all = reinterpret_cast<unsigned short*>(xt + kXRows * dm * RB);
  for (int e = 2; e <= dm; ++e) {
    const int np = e * (e - 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      int j = 0, rem = p;
      while (rem >= e - 1 - j) {
        rem -= e - 1 - j;
        ++j;
      }
      pairs_all[e * (e - 1) * (e - 2) / 6 + p] = (unsigned short)((j << 8) | (j + 1 + rem));
    }
  }
  __syncthreads();
  const BatchState* bs = B.bs;
  const int cur = bs->parity;
  const double* C = B.c[cur];
  const double* H = B.h[cur];
  const int32_t* rid = B.rid[cur];
  const int tid = threadIdx.x;
  auto tab = [&](int row, int j) -> float { return xt[(row * dm + j) * RB + tid]; };
  const float l2 = (float)B.lam2, l3 = (float)B.lam3, l5 = (float)B.lam5;
  // this family's regions: one contiguous range (the batch is in family order)
  const long long r_lo = bs->fam_off[cur][FAM], r_hi = bs->fam_off[cur][FAM + 1];
  for (long long tile = blockIdx.x; r_lo + tile * RB < r_hi; tile += gridDim.x) {
    const long long r = r_lo + tile * RB + tid;
    if (r >= r_hi) break;
    const BatchItem& it = B.items[rid[r]];
    if (it.paused) continue;  // carried over with its outputs
    const int d = it.P.d;
    for (int k = 0; k < d; ++k)
      mixed_coord_rows(C[(int64_t)k * B.ld + r], H[(int64_t)k * B.ld + r], l2, l3, l5,
                       xt + k * RB + tid, dm * RB);
    auto cval = [&](int k) { return C[(int64_t)k * B.ld + r]; };
    auto hval = [&](int k) { return H[(int64_t)k * B.ld + r]; };
    RegionSums o;
    switch (d) {
      case 3: region_mixed_walk<FAM, 3>(it.Pf, tab, B.ratio, o); break;
      case 4: region_mixed_walk<FAM, 4>(it.Pf, tab, B.ratio, o); break;
      case 5: region_mixed_walk<FAM, 5>(it.Pf, tab, B.ratio, o); break;
      case 6: region_mixed_walk<FAM, 6>(it.Pf, tab, B.ratio, o); break;
      case 7: region_mixed_walk<FAM, 7>(it.Pf, tab, B.ratio, o); break;
      case 8: region_mixed_walk<FAM, 8>(it.Pf, tab, B.ratio, o); break;
      case 9: region_mixed_walk<FAM, 9>(it.Pf, tab, B.ratio, o); break;
      case 10: region_mixed_walk<FAM, 10>(it.Pf, tab, B.ratio, o); break;
      case 11: region_mixed_walk<FAM, 11>(it.Pf, tab, B.ratio, o); break;
      case 12: region_mixed_walk<FAM, 12>(it.Pf, tab, B.ratio, o); break;
      default:
        region_mixed_flat<FAM>(it.Pf, d, pairs_all + d * (d - 1) * (d - 2) / 6, tab, B.ratio, o);
        break;
    }
    region_finish64(o, d, it.w7, it.w5, B.estimator ? it.nw : nullptr, it.vol_omega, cval, hval,
                    B.i7[cur] + r, B.err[cur] + r, B.vf[cur] + r, B.axis[cur] + r);
  }
}

template <int FAM>
cudaError_t batch_launch_rule_mixed_family(const BatchArgs& B, int grid, cudaStream_t s) {
  const size_t smem = batch_rule_mixed_smem(B.dmax);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_rule_mixed<FAM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_batch_rule_mixed<FAM><<<grid, kBatchRuleBlock, smem, s>>>(B);
  return cudaGetLastError();
}

template <int FAM>
int batch_rule_mixed_max_blocks_family(int dmax) {
  int nb = 0;
  const size_t smem = batch_rule_mixed_smem(dmax);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_batch_rule_mixed<FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_rule_mixed<FAM>,
                                                    kBatchRuleBlock, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

#define GMQ_DEFINE_BATCH_MIXED_FAMILY(FAMV)                                                 \
  template cudaError_t batch_launch_rule_mixed_family<FAMV>(const BatchArgs&, int,           \
                                                            cudaStream_t);                   \
  template int batch_rule_mixed_max_blocks_family<FAMV>(int);

}  // namespace gmq
