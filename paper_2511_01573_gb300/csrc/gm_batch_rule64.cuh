// gm_batch_rule64.cuh -- FP64 rule evaluation of the batched form, one
// kernel per integrand family (instantiated with the other per-family
// kernels in gm_rule_inst.cu).  The batch is in family order, so each
// family's regions are one contiguous range of the list; a launch walks its
// family's range on a persistent grid with T = bs->lanes lanes per region
// (1, 4, 32 or a 128-thread block; chosen per sweep, never changing a
// result) and the single-integral FP64 path's per-region code
// (gm_region64.cuh) specialised for the family, so every region gets the
// bits gmq_integrate gives it, from a kernel whose registers and code are
// those of its own integrand rather than of all seven.
#pragma once

#include "gm_batch.cuh"
#include "gm_region64.cuh"

namespace gmq {

template <int FAM, int T>
__device__ __forceinline__ void batch_rule64_lanes(const BatchArgs& B, double* smem,
                                                   const unsigned short* pairs_all) {
  constexpr int RPB = kBatchRuleBlock / T;  // regions per tile
  const BatchState* bs = B.bs;
  const int cur = bs->parity;
  const long long r_lo = bs->fam_off[cur][FAM], r_hi = bs->fam_off[cur][FAM + 1];
  const double* C = B.c[cur];
  const double* H = B.h[cur];
  const int32_t* rid = B.rid[cur];
  const int64_t ld = B.ld;
  const int tid = threadIdx.x;
  const int g = tid / T, lane = tid & (T - 1);
  const unsigned mask = group_mask<T>();
  double* wsp = smem + g;  // this group's region workspace, entries RPB apart
  for (long long tile = blockIdx.x; r_lo + tile * RPB < r_hi; tile += gridDim.x) {
    const long long r = r_lo + tile * RPB + g;
    if (r >= r_hi) break;  // so are the group's later tiles
    group_sync<T>(mask);   // the group is done with the previous region's workspace
    const BatchItem& it = B.items[rid[r]];
    if (it.paused) continue;  // carried over with last sweep's outputs
    const int d = it.P.d;
    auto ch = [&](int k, double& c, double& h) {
      c = C[(int64_t)k * ld + r];
      h = H[(int64_t)k * ld + r];
    };
    RegionSums o;
    region_sums64<FAM, T>(it.P, d, pairs_all + batch_pairs_offset(d), ch, B.lam2, B.lam3,
                          B.lam5, wsp, RPB, B.ratio, o);
    if (lane == 0)
      region_finish64(
          o, d, it.w7, it.w5, B.estimator ? it.nw : nullptr, it.vol_omega,
          [&](int k) { return C[(int64_t)k * ld + r]; },
          [&](int k) { return H[(int64_t)k * ld + r]; }, B.i7[cur] + r, B.err[cur] + r,
          B.vf[cur] + r, B.axis[cur] + r);
  }
}

// Rule evaluation of family FAM's regions of the current list: persistent
// grid of kBatchRuleBlock-thread blocks, T = bs->lanes lanes per region.
template <int FAM>
__global__ void __launch_bounds__(kBatchRuleBlock) k_batch_rule64(const BatchArgs B) {
  extern __shared__ __align__(16) double smem[];
  const int dm = B.dmax;
  unsigned short* pairs_all = reinterpret_cast<unsigned short*>(smem + batch_rule_doubles_max(dm));
  for (int e = 2; e <= dm; ++e) {
    const int np = e * (e - 1) / 2;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      int j = 0, rem = p;
      while (rem >= e - 1 - j) {
        rem -= e - 1 - j;
        ++j;
      }
      pairs_all[batch_pairs_offset(e) + p] = (unsigned short)((j << 8) | (j + 1 + rem));
    }
  }
  __syncthreads();
  const int lanes = B.bs->lanes;
  if (lanes == 128)
    batch_rule64_lanes<FAM, 128>(B, smem, pairs_all);
  else if (lanes == 32)
    batch_rule64_lanes<FAM, 32>(B, smem, pairs_all);
  else if (lanes == 4)
    batch_rule64_lanes<FAM, 4>(B, smem, pairs_all);
  else
    batch_rule64_lanes<FAM, 1>(B, smem, pairs_all);
}

template <int FAM>
cudaError_t batch_launch_rule64_family(const BatchArgs& B, int grid, cudaStream_t s) {
  const size_t smem = batch_rule_smem(B.dmax);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_rule64<FAM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_batch_rule64<FAM><<<grid, kBatchRuleBlock, smem, s>>>(B);
  return cudaGetLastError();
}

template <int FAM>
int batch_rule64_max_blocks_family(int dmax) {
  int nb = 0;
  const size_t smem = batch_rule_smem(dmax);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_batch_rule64<FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_rule64<FAM>, kBatchRuleBlock,
                                                    smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

#define GMQ_DEFINE_BATCH_RULE64_FAMILY(FAMV)                                                \
  template cudaError_t batch_launch_rule64_family<FAMV>(const BatchArgs&, int, cudaStream_t); \
  template int batch_rule64_max_blocks_family<FAMV>(int);

}  // namespace gmq
