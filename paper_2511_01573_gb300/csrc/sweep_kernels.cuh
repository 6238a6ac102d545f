// sweep_kernels.cuh -- launchers of the per-sweep kernels (sums, classify,
// split, partition) defined in sweep_kernels.cu.
#pragma once

#include "gmq_common.cuh"

namespace gmq {

struct PartArgs {
  int32_t d;
  int32_t s;
  int64_t n;  // s^d
  double lo[GMQ_MAX_DIM];
  double h[GMQ_MAX_DIM];  // (hi - lo) / (2 s), computed on the host
  double* c_out;
  double* h_out;
  int64_t ld;
};

cudaError_t launch_sum_status(const SweepArgs& S, cudaStream_t s);
cudaError_t launch_classify(const SweepArgs& S, cudaStream_t s);
cudaError_t launch_split(const SweepArgs& S, cudaStream_t s);
cudaError_t launch_partition(const PartArgs& P, cudaStream_t s);
cudaError_t launch_tree_sum(const double* v, int64_t n, double* blk, DevStatus* st, double* out,
                            cudaStream_t s);
// blk: rows * ceil(n / kTile) doubles; tickets: rows zeroed counters.
cudaError_t launch_rows_tree_sum(const double* v, int64_t ldv, int64_t n, int rows, double* blk,
                                 unsigned* tickets, double* out, cudaStream_t s);

// Issue-rate probe (fma_probe.cu): `blocks` blocks of kProbeBlock threads
// running chains of one operation (op 0 fused multiply-add, 1 add, 2
// multiply); sink holds blocks * kProbeBlock elements (double if fp64, else
// float).  fma_probe_lane_fmas: the lane operations one launch performs.
constexpr int kProbeBlock = 256;
cudaError_t launch_fma_probe(int fp64, int op, int blocks, int64_t iters, void* sink,
                             cudaStream_t s);
int64_t fma_probe_lane_fmas(int blocks, int64_t iters);

}  // namespace gmq
