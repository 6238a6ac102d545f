// gmq_common.cuh -- internal types and device helpers shared by the kernels
// of the GB300 adaptive Genz-Malik quadrature library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gmq.h"

namespace gmq {

// Regions per tile of the sweep kernels (classify, split, sums): one region
// per thread, 1024 threads.  A power of two, so that tile sums are complete
// subtrees of the pairwise summation tree.
constexpr int kTile = 1024;

// Threads per block of the rule kernel.
constexpr int kRuleBlock = 128;

// Family parameters as the device functors use them.  Filled on the host
// from gmq_problem: a, u as given; b is a per-axis constant of the family
// (a^-2 for the product peak, a^2 for the Gaussian); c0 a scalar
// (2 pi u_1 for the oscillatory family).
struct FamParams {
  int32_t d;
  int32_t family;
  double c0;
  double a[GMQ_MAX_DIM];
  double u[GMQ_MAX_DIM];
  double b[GMQ_MAX_DIM];
};

// Rule constants for dimension d (Genz & Malik 1980; paper Sec. 2).
struct RuleConst {
  double lam2, lam3, lam5;  // generators (lambda4 == lambda3)
  double w7[5];             // degree-7 class weights (unit volume)
  double w5[5];             // embedded degree-5 class weights
  double ratio;             // lambda2^2 / lambda3^2 = 1/7
  double vol_omega;         // prod_k (hi_k - lo_k)
  int64_t nodes;            // 2^d + 2d^2 + 2d + 1
  int32_t estimator;        // gmq_estimator
  double nw[20];            // null-rule weights (GMQ_EST_NULL_RULES), 4 x 5
};

struct RuleArgs {
  const double* c;
  const double* h;
  int64_t ld;
  int64_t n;
  double* i7;
  double* err;
  double* volfrac;   // may be null
  uint8_t* axis;
  FamParams P;
  RuleConst R;
  int32_t nodewise;  // FP64 Genz-Malik kernels: 1 = evaluate f node by node (GMQ_EVAL_NODEWISE)
};

// Device-side state of one integration, updated by the sweep kernels and
// copied to the host once per sweep.
struct DevStatus {
  double I_ret, E_ret;   // running sums of retired regions
  double I, E, budget;   // this sweep's global estimates
  double ret_i, ret_e;   // this sweep's retired sums
  long long n_split;     // regions split in this sweep
  long long n_leaves;    // regions recorded in the final-partition list
  long long leaf_base;   // n_leaves before this sweep's retired regions
  int flags;             // kConverged | kNonfinite | kCap | kDone ...
  unsigned ticket_sum;   // last-block counters (reset by the last block)
  unsigned ticket_cls;
  int pad;
};
enum {
  kConverged = 1,
  kNonfinite = 2,
  kCapExceeded = 4,
  kAllRetired = 8,
  kDone = 16,
  kLastSweep = 32,    // the sweep limit is reached: stop after the sums
  kLeafOverflow = 64  // the final-partition list is full
};

// Parameters of the sum / classify / split kernels of one sweep.
struct SweepArgs {
  int64_t n;
  int32_t d;
  int32_t classifier;
  double rel_tol, abs_tol;
  int64_t cap;             // capacity of the output arrays
  const double* c;
  const double* h;
  int64_t ld;
  double* c_out;
  double* h_out;
  int64_t ld_out;
  const double* i7;
  const double* err;
  const double* volfrac;
  const uint8_t* axis;
  uint8_t* flags;
  int* blk_count;          // per tile: regions split
  long long* blk_off;      // per tile: exclusive prefix of blk_count
  double* blk_a;           // per tile partial sums (two arrays)
  double* blk_b;
  const double* budget_ptr;  // device budget (integrate path) or null
  double budget_val;         // host budget (step-level path)
  double guard;              // round-off guard factor g*u: retire if err <= guard |I7|
  int last_sweep;            // 1: this is the last sweep the loop may run
  int keep;                  // 1: record retired regions in the leaf list
  double* c_leaf;            // final-partition list (keep == 1)
  double* h_leaf;
  int64_t ld_leaf;
  int64_t leaf_cap;
  DevStatus* st;
};

// Pairwise-tree sum over the threads of a block, one value per thread,
// blockDim.x a power of two <= 1024: value of thread t is element t.
// Returns the total in every thread.  scratch: >= 32 doubles of shared memory.
__device__ __forceinline__ double block_tree_sum(double v, double* scratch) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  // adjacent pairs first: offsets 1, 2, 4, 8, 16 build the tree of the warp
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    double o = __shfl_down_sync(0xffffffffu, v, off);
    v = v + o;  // lanes whose partner lies outside keep garbage in unused slots only
  }
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  const unsigned nw = blockDim.x >> 5;
  double w = 0.0;
  if (warp == 0) {
    w = lane < nw ? scratch[lane] : 0.0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      double o = __shfl_down_sync(0xffffffffu, w, off);
      w = w + o;
    }
    if (lane == 0) scratch[32] = w;
  }
  __syncthreads();
  double tot = scratch[32];
  __syncthreads();
  return tot;
}

}  // namespace gmq
