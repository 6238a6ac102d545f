// gm_batch.cuh -- data structures and launchers of the batched form
// (gmq_integrate_batch): many integrals advanced together, one sweep per
// iteration of a device-side loop (kernels in gm_batch.cu).
#pragma once

#include "gmq_common.cuh"
#include "gmq_families.cuh"
#include "gm_region64.cuh"

namespace gmq {

constexpr int kBatchRuleBlock = 128;  // threads per block of the rule kernel

// Per-integral descriptor (problem, rule constants) and loop state.
struct BatchItem {
  FamParams P;
  SmemParams<float> Pf;    // the parameters rounded to FP32 (mixed form)
  double w7[5], w5[5];
  double nw[20];           // null-rule weights (GMQ_EST_NULL_RULES)
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
  long long nnext;         // regions of the next list (set by the scan)
  unsigned tk_sum, tk_cls; // tiles of this integral done in the sums / classify kernels
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
  int lanes;               // lanes per region of this sweep's rule kernel (1, 4, 32, 128)
  int lane_sweeps[4];      // sweeps run with 1, 4, 32 and 128 lanes per region
  long long n_tiles;       // tiles of the current list (kSegTile regions, one integral each)
  long long n_tiles_next;  // tiles of the next list
  long long fam_off[2][8]; // first region of each family in either list; [p][7] = length
  long long rule_regions;     // regions the rule kernels evaluated (work later
                              // dropped by evictions included)
  long long carried_regions;  // regions of paused integrals carried over unchanged
  long long list_regions;     // sum over sweeps of the list length
  long long carried_cur;      // regions of the current list carried over (not evaluated)
  long long carried_next;     // regions this sweep's scan carries into the next list
};

// The per-integral sweep kernels work on tiles of kSegTile consecutive
// regions of one integral (its last tile may be short): tile t of the list
// of parity p belongs to the integral i with tile_off[p][i] <= t <
// tile_off[p][i + 1].
constexpr int kSegBlock = 1024;           // threads of the tile kernels
constexpr int kSegTile = 4 * kSegBlock;   // regions per tile (4 per thread)

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
  // rule outputs of both lists (a paused integral's outputs move with its
  // regions, and its regions are not evaluated again)
  double* i7[2];
  double* err[2];
  double* vf[2];
  uint8_t* axis[2];
  uint8_t* flags;
  int dmax;
  int classifier;
  int estimator;           // gmq_estimator of every integral of the batch
  double guard;
  double lam2, lam3, lam5, ratio;
  cudaGraphConditionalHandle cond;
  int use_cond;
  // lanes per region of the rule kernel: forced_lanes if nonzero, else 1
  // for lists of at least lanes_t1 regions, 4 from lanes_t4, 32 from
  // lanes_t32, 128 (a block) below
  int forced_lanes;
  long long lanes_t1, lanes_t4, lanes_t32;
  // tiles: per-integral tile offsets of both lists (count + 1 entries each)
  // and per-tile partial results
  long long* tile_off[2];
  double* tile_a;
  double* tile_b;
  long long* tile_cnt;
  long long* tile_pos;
  int tile_grid;           // blocks of the persistent tile kernels
  int fam_item_lo[8];      // items are in family order: family f is items
                           // [fam_item_lo[f], fam_item_lo[f + 1]), [7] = count
};

__host__ __device__ inline int batch_lanes_for(const BatchArgs& B, long long n) {
  if (B.forced_lanes) return B.forced_lanes;
  return n >= B.lanes_t1 ? 1 : (n >= B.lanes_t4 ? 4 : (n >= B.lanes_t32 ? 32 : 128));
}


// Doubles of the FP64 rule kernel's per-block region workspaces for T lanes
// per region: 128 / T workspaces of the largest layout over dimensions
// 1 .. dmax (gm_region64.cuh; flag masks included for every family); the
// kernel sizes its shared memory for the largest over T.
__host__ __device__ constexpr long long batch_rule_doubles(int dmax, int T) {
  return (long long)sep_words_max(dmax, true, T > 1) * (kBatchRuleBlock / T);
}
__host__ __device__ constexpr long long batch_rule_doubles_max(int dmax) {
  long long m = batch_rule_doubles(dmax, 1);
  if (batch_rule_doubles(dmax, 4) > m) m = batch_rule_doubles(dmax, 4);
  if (batch_rule_doubles(dmax, 32) > m) m = batch_rule_doubles(dmax, 32);
  if (batch_rule_doubles(dmax, 128) > m) m = batch_rule_doubles(dmax, 128);
  return m;
}

// Pair tables of every dimension 2 .. dmax, one after the other: the table
// of dimension d starts at entry d (d - 1) (d - 2) / 6.
__host__ __device__ constexpr int batch_pairs_offset(int d) { return d * (d - 1) * (d - 2) / 6; }

// Shared memory of the FP64 rule kernel for the largest dimension.
size_t batch_rule_smem(int dmax);
cudaError_t batch_launch_partition(const BatchArgs& B, cudaStream_t s);
// FP64 rule evaluation of the current list's regions of family FAM
// (gm_batch_rule64.cuh; one launch per family present in the batch,
// persistent grid, bs->lanes lanes per region).
template <int FAM>
cudaError_t batch_launch_rule64_family(const BatchArgs& B, int grid, cudaStream_t s);
template <int FAM>
int batch_rule64_max_blocks_family(int dmax);
// Mixed form: rule evaluation of the current list's regions of family FAM
// (gm_batch_mixed.cuh; one launch per family present in the batch).
template <int FAM>
cudaError_t batch_launch_rule_mixed_family(const BatchArgs& B, int grid, cudaStream_t s);
template <int FAM>
int batch_rule_mixed_max_blocks_family(int dmax);
// Fill list 0 positions [n0, n) with copies of its regions [0, n0).
cudaError_t batch_launch_tile(const BatchArgs& B, long long n0, long long n, cudaStream_t s);
// Sums, classification, scan, split and loop advance of one sweep.
cudaError_t batch_launch_rest(const BatchArgs& B, cudaStream_t s);

}  // namespace gmq
