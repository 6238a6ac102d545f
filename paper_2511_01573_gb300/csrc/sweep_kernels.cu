// sweep_kernels.cu -- the per-sweep kernels around the rule evaluation
// (paper Sec. 3 loop, Fig. 1a):
//   k_sum_status  global sums I = I_ret + sum I_r, eps = E_ret + sum eps_r,
//                 budget max(abs_tol, rel_tol |I|) and the convergence test
//                 (paper Sec. 4 stopping rule);
//   k_classify    retire/split decision per region (heuristic classifier and
//                 round-off guards, paper Sec. 3), retired sums, per-tile
//                 split counts and, in the last tile to finish, the scan of
//                 the tile counts and the status update;
//   k_split       bisection of the split regions into the output list
//                 (left children first, then right children), compacted by
//                 the scan;
//   k_partition   the initial uniform partition (paper Sec. 3).
// All sums use the pairwise tree over the list zero-padded to a power of
// two: a tile of 1024 regions is a complete subtree, the last block to
// finish sums the tile results with the same tree.  No floating-point
// atomics: the result does not depend on scheduling.
#include "gmq_common.cuh"
#include "sweep_kernels.cuh"

namespace gmq {

namespace {

// Pairwise-tree sum of v[0..count) in one block of kTile threads.
__device__ double tree_sum_global(const double* v, int64_t count, double* scratch,
                                  double* tile_sums) {
  const int tid = threadIdx.x;
  if (count <= kTile) {
    return block_tree_sum(tid < count ? v[tid] : 0.0, scratch);
  }
  const int64_t nt = (count + kTile - 1) / kTile;  // <= kTile by construction
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t i = t * kTile + tid;
    const double s = block_tree_sum(i < count ? v[i] : 0.0, scratch);
    if (tid == 0) tile_sums[t] = s;
  }
  __syncthreads();
  return block_tree_sum(tid < nt ? tile_sums[tid] : 0.0, scratch);
}

// Exclusive scan of in[0..count) (int) into out (long long) by one block;
// returns the total.
__device__ long long block_exclusive_scan(const int* in, long long* out, int64_t count,
                                          long long* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  long long carry = 0;
  for (int64_t base = 0; base < count; base += kTile) {
    const int64_t i = base + tid;
    long long v = i < count ? (long long)in[i] : 0;
    // inclusive warp scan
    long long x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long w = wsum[lane];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      wsum[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const long long before = (warp > 0 ? wsum[warp - 1] : 0) + (x - v);
    if (i < count) out[i] = carry + before;
    const long long tot = wsum[31];
    __syncthreads();
    carry += tot;
  }
  return carry;
}

}  // namespace

__global__ void __launch_bounds__(kTile) k_sum_status(const SweepArgs S) {
  __shared__ double scratch[33];
  __shared__ double tile_sums[kTile];
  __shared__ int is_last;
  if (S.st->flags & kDone) return;
  const int64_t r = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const double a = r < S.n ? S.i7[r] : 0.0;
  const double b = r < S.n ? S.err[r] : 0.0;
  const double ta = block_tree_sum(a, scratch);
  const double tb = block_tree_sum(b, scratch);
  if (threadIdx.x == 0) {
    S.blk_a[blockIdx.x] = ta;
    S.blk_b[blockIdx.x] = tb;
    __threadfence();
    const unsigned t = atomicAdd(&S.st->ticket_sum, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const double A = tree_sum_global(S.blk_a, gridDim.x, scratch, tile_sums);
  const double B = tree_sum_global(S.blk_b, gridDim.x, scratch, tile_sums);
  if (threadIdx.x == 0) {
    DevStatus* st = S.st;
    st->ticket_sum = 0u;
    const double I = __dadd_rn(st->I_ret, A);
    const double E = __dadd_rn(st->E_ret, B);
    const double budget = fmax(S.abs_tol, __dmul_rn(S.rel_tol, fabs(I)));
    st->I = I;
    st->E = E;
    st->budget = budget;
    int f = st->flags;
    if (!isfinite(I) || !isfinite(E))
      f |= kNonfinite | kDone;
    else if (E <= budget)
      f |= kConverged | kDone;
    else if (S.last_sweep)
      f |= kLastSweep | kDone;
    st->flags = f;
  }
}

__global__ void __launch_bounds__(kTile) k_classify(const SweepArgs S) {
  __shared__ double scratch[33];
  __shared__ double tile_sums[kTile];
  __shared__ long long wsum[32];
  __shared__ int is_last;
  if (S.st->flags & kDone) return;
  const int64_t r = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const double budget = S.budget_ptr ? *S.budget_ptr : S.budget_val;
  int split = 0;
  double ri = 0.0, re = 0.0;
  if (r < S.n) {
    const double i7 = S.i7[r];
    const double e = S.err[r];
    const uint8_t ax = S.axis[r];
    const double thr = (S.classifier == GMQ_LOCAL_REL) ? __dmul_rn(S.rel_tol, fabs(i7))
                                                       : __dmul_rn(budget, S.volfrac[r]);
    const double guard = __dmul_rn(S.guard, fabs(i7));
    const bool retire = (e <= thr) || (e <= guard) || (ax & 0x80);
    split = retire ? 0 : 1;
    if (retire) {
      ri = i7;
      re = e;
    }
    S.flags[r] = (uint8_t)split;
  }
  const int cnt = __syncthreads_count(split);
  const double ta = block_tree_sum(ri, scratch);
  const double tb = block_tree_sum(re, scratch);
  if (threadIdx.x == 0) {
    S.blk_count[blockIdx.x] = cnt;
    S.blk_a[blockIdx.x] = ta;
    S.blk_b[blockIdx.x] = tb;
    __threadfence();
    const unsigned t = atomicAdd(&S.st->ticket_cls, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const long long total = block_exclusive_scan(S.blk_count, S.blk_off, gridDim.x, wsum);
  const double A = tree_sum_global(S.blk_a, gridDim.x, scratch, tile_sums);
  const double B = tree_sum_global(S.blk_b, gridDim.x, scratch, tile_sums);
  if (threadIdx.x == 0) {
    DevStatus* st = S.st;
    st->ticket_cls = 0u;
    st->ret_i = A;
    st->ret_e = B;
    st->I_ret = __dadd_rn(st->I_ret, A);
    st->E_ret = __dadd_rn(st->E_ret, B);
    st->n_split = total;
    int f = st->flags;
    if (total == 0) {
      f |= kAllRetired | kDone;
    } else if (2 * total > S.cap) {
      f |= kCapExceeded | kDone;
    } else if (S.keep) {
      // the split kernel appends this sweep's retired regions to the leaves
      const long long nl = st->n_leaves + (S.n - total);
      if (nl > S.leaf_cap) {
        f |= kLeafOverflow | kDone;
      } else {
        st->leaf_base = st->n_leaves;
        st->n_leaves = nl;
      }
    }
    st->flags = f;
  }
}

__global__ void __launch_bounds__(kTile) k_split(const SweepArgs S) {
  __shared__ int wcount[32];
  if (S.st->flags & kDone) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r = (int64_t)blockIdx.x * kTile + tid;
  const int f = (r < S.n) ? (int)S.flags[r] : 0;
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) wcount[warp] = __popc(bal);
  __syncthreads();
  int wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += wcount[w];
  if (r >= S.n) return;
  // split regions before r in the whole list
  const long long pos = S.blk_off[blockIdx.x] + wpre + __popc(bal & ((1u << lane) - 1u));
  if (!f) {
    if (S.keep) {
      // retired: append to the final-partition list after the earlier
      // retired regions of this sweep (r - pos of them)
      const long long leaf = S.st->leaf_base + (r - pos);
      for (int k = 0; k < S.d; ++k) {
        S.c_leaf[(int64_t)k * S.ld_leaf + leaf] = S.c[(int64_t)k * S.ld + r];
        S.h_leaf[(int64_t)k * S.ld_leaf + leaf] = S.h[(int64_t)k * S.ld + r];
      }
    }
    return;
  }
  const long long ns = S.st->n_split;
  const int ax = S.axis[r] & 0x7f;
  for (int k = 0; k < S.d; ++k) {
    const double c = S.c[(int64_t)k * S.ld + r];
    const double h = S.h[(int64_t)k * S.ld + r];
    double cl = c, cr = c, hc = h;
    if (k == ax) {
      hc = __dmul_rn(0.5, h);
      cl = __dsub_rn(c, hc);
      cr = __dadd_rn(c, hc);
    }
    S.c_out[(int64_t)k * S.ld_out + pos] = cl;
    S.h_out[(int64_t)k * S.ld_out + pos] = hc;
    S.c_out[(int64_t)k * S.ld_out + ns + pos] = cr;
    S.h_out[(int64_t)k * S.ld_out + ns + pos] = hc;
  }
}

__global__ void k_partition(const PartArgs P) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.n) return;
  int64_t rem = q;
  for (int k = 0; k < P.d; ++k) {
    const int64_t i = rem % P.s;
    rem /= P.s;
    const double hk = P.h[k];
    P.c_out[(int64_t)k * P.ld + q] = __dadd_rn(P.lo[k], __dmul_rn((double)(2 * i + 1), hk));
    P.h_out[(int64_t)k * P.ld + q] = hk;
  }
}

// Standalone pairwise sum into st->I (for the step-level tree-sum call).
__global__ void __launch_bounds__(kTile) k_tree_sum(const double* v, int64_t n, double* blk,
                                                    DevStatus* st, double* out) {
  __shared__ double scratch[33];
  __shared__ double tile_sums[kTile];
  __shared__ int is_last;
  const int64_t r = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const double t = block_tree_sum(r < n ? v[r] : 0.0, scratch);
  if (threadIdx.x == 0) {
    blk[blockIdx.x] = t;
    __threadfence();
    const unsigned k = atomicAdd(&st->ticket_sum, 1u);
    is_last = (k == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const double s = tree_sum_global(blk, gridDim.x, scratch, tile_sums);
  if (threadIdx.x == 0) {
    st->ticket_sum = 0u;
    *out = s;
  }
}

// Pairwise-tree sum of every row of v ([rows][ldv], n values per row):
// blockIdx.y is the row; the last tile of a row to finish writes out[row].
__global__ void __launch_bounds__(kTile) k_rows_tree_sum(const double* v, int64_t ldv, int64_t n,
                                                         double* blk, unsigned* tickets,
                                                         double* out) {
  __shared__ double scratch[33];
  __shared__ double tile_sums[kTile];
  __shared__ int is_last;
  const int row = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * kTile + threadIdx.x;
  const double t = block_tree_sum(r < n ? v[(int64_t)row * ldv + r] : 0.0, scratch);
  double* rb = blk + (int64_t)row * gridDim.x;
  if (threadIdx.x == 0) {
    rb[blockIdx.x] = t;
    __threadfence();
    const unsigned k = atomicAdd(&tickets[row], 1u);
    is_last = (k == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const double s = tree_sum_global(rb, gridDim.x, scratch, tile_sums);
  if (threadIdx.x == 0) {
    tickets[row] = 0u;
    out[row] = s;
  }
}

cudaError_t launch_rows_tree_sum(const double* v, int64_t ldv, int64_t n, int rows, double* blk,
                                 unsigned* tickets, double* out, cudaStream_t s) {
  int64_t blocks = (n + kTile - 1) / kTile;
  if (blocks == 0) blocks = 1;
  k_rows_tree_sum<<<dim3((unsigned)blocks, (unsigned)rows), kTile, 0, s>>>(v, ldv, n, blk, tickets,
                                                                          out);
  return cudaGetLastError();
}

cudaError_t launch_sum_status(const SweepArgs& S, cudaStream_t s) {
  const int64_t blocks = (S.n + kTile - 1) / kTile;
  if (blocks == 0) return cudaSuccess;
  k_sum_status<<<(unsigned)blocks, kTile, 0, s>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_classify(const SweepArgs& S, cudaStream_t s) {
  const int64_t blocks = (S.n + kTile - 1) / kTile;
  if (blocks == 0) return cudaSuccess;
  k_classify<<<(unsigned)blocks, kTile, 0, s>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_split(const SweepArgs& S, cudaStream_t s) {
  const int64_t blocks = (S.n + kTile - 1) / kTile;
  if (blocks == 0) return cudaSuccess;
  k_split<<<(unsigned)blocks, kTile, 0, s>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_partition(const PartArgs& P, cudaStream_t s) {
  const int64_t blocks = (P.n + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  k_partition<<<(unsigned)blocks, 256, 0, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_tree_sum(const double* v, int64_t n, double* blk, DevStatus* st, double* out,
                            cudaStream_t s) {
  int64_t blocks = (n + kTile - 1) / kTile;
  if (blocks == 0) blocks = 1;
  k_tree_sum<<<(unsigned)blocks, kTile, 0, s>>>(v, n, blk, st, out);
  return cudaGetLastError();
}

}  // namespace gmq
