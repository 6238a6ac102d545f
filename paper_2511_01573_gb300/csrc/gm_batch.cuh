// gm_batch.cuh -- data structures and launchers of the batched form
// (gmq_integrate_batch): many integrals advanced together, one sweep per
// iteration of a device-side loop (kernels in gm_batch.cu).
#pragma once

#include "gmq_common.cuh"

namespace gmq {

constexpr int kBatchRuleBlock = 128;  // threads per block of the rule kernel

// Per-integral descriptor (problem, rule constants) and loop state.
struct BatchItem {
  FamParams P;
  double w7[5], w5[5];
  double vol_omega;
  double rel_tol, abs_tol;
  double lo[GMQ_MAX_DIM];
  double h0[GMQ_MAX_DIM];  // initial half-widths (hi - lo) / (2 s)
  int32_t s;               // initial splits per axis
  int32_t nodes;           // 2^d + 2d^2 + 2d + 1
  long long cap;           // per-integral region cap
  // state
  double I_ret, E_ret, I, E, budget;
  long long off, n, noff;  // current segment, next segment offset
  long long n_split;
  long long regions;       // regions evaluated
  double ret_i, ret_e;     // this sweep's retired sums, committed when it splits
  long long n0;            // regions of the initial partition (s^d)
  int iters;
  int flags;               // kConverged | kNonfinite | kCapExceeded | ...
  int paused;              // 1: this sweep's split did not fit in the pool
  int deferred;            // 1: evicted, holds no regions, waits for room
  int restart;             // 1: the split kernel writes the initial partition
  int pad;
};

// Batch-wide loop state.
struct BatchState {
  long long n_total;       // regions in the current list
  long long n_next;        // regions in the next list
  int parity;              // 0: list A is current, 1: list B
  int active;              // integrals still running
  int sweep;
  int max_iters;           // per-integral sweep limit
  int max_sweeps;          // bound of the device loop (pauses add sweeps)
  int pauses;              // integral-sweeps paused for lack of pool space
  int evictions;           // integrals evicted to make room (restarted later)
  int lanes;               // lanes per region of this sweep's rule kernel (1, 4, 32)
  int lane_sweeps[3];      // sweeps run with 1, 4 and 32 lanes per region
};

// Arguments of every batch kernel (passed by value).
struct BatchArgs {
  BatchItem* items;
  int32_t count;
  BatchState* bs;
  double* c[2];
  double* h[2];
  int32_t* rid[2];
  int64_t ld;
  int64_t pool_cap;
  double* i7;
  double* err;
  double* vf;
  uint8_t* axis;
  uint8_t* flags;
  int dmax;
  int classifier;
  double guard;
  double lam2, lam3, lam5, ratio;
  cudaGraphConditionalHandle cond;
  int use_cond;
  // lanes per region of the rule kernel: forced_lanes if nonzero, else 1
  // for lists of at least lanes_t1 regions, 4 from lanes_t4, 32 below
  int forced_lanes;
  long long lanes_t1, lanes_t4;
};

__host__ __device__ inline int batch_lanes_for(const BatchArgs& B, long long n) {
  if (B.forced_lanes) return B.forced_lanes;
  return n >= B.lanes_t1 ? 1 : (n >= B.lanes_t4 ? 4 : 32);
}


// Shared memory of the rule kernel for the largest dimension.
size_t batch_rule_smem(int dmax);
// Resident blocks per SM of the rule kernel.
int batch_rule_max_blocks(int dmax);
cudaError_t batch_launch_partition(const BatchArgs& B, cudaStream_t s);
// Rule evaluation of every region of the current list (persistent grid,
// bs->lanes lanes per region).
cudaError_t batch_launch_rule(const BatchArgs& B, int grid, cudaStream_t s);
// Fill list 0 positions [n0, n) with copies of its regions [0, n0).
cudaError_t batch_launch_tile(const BatchArgs& B, long long n0, long long n, cudaStream_t s);
// Sums, classification, scan, split and loop advance of one sweep.
cudaError_t batch_launch_rest(const BatchArgs& B, cudaStream_t s);

}  // namespace gmq
