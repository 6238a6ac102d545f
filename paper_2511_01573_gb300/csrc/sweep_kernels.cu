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
#include <cstdint>

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

// The same trees with a quarter of the threads: kQuad threads, thread t
// holding the 4 consecutive values 4t .. 4t + 3 of a tile.  Its
// ((v0 + v1) + (v2 + v3)) are the first two levels of the tile's pairwise
// tree and block_tree_sum adds the rest, so a tile sum is bit-identical to
// the kTile-thread form.
constexpr int kQuad = kTile / 4;

__device__ __forceinline__ double tile_sum4(const double* v, int64_t base, int64_t count,
                                            double* scratch) {
  const int64_t i = base + 4 * (int64_t)threadIdx.x;
  const double a = i < count ? v[i] : 0.0, b = i + 1 < count ? v[i + 1] : 0.0;
  const double c = i + 2 < count ? v[i + 2] : 0.0, d = i + 3 < count ? v[i + 3] : 0.0;
  return block_tree_sum((a + b) + (c + d), scratch);
}

// tree_sum_global for blocks of kQuad threads; the partials were written by
// other blocks of this launch (read through L2).
__device__ double tree_sum_global4(const double* v, int64_t count, double* scratch,
                                   double* tile_sums) {
  if (count <= kTile) {
    const int64_t i = 4 * (int64_t)threadIdx.x;
    double q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = i + k < count ? __ldcg(v + i + k) : 0.0;
    return block_tree_sum((q[0] + q[1]) + (q[2] + q[3]), scratch);
  }
  const int64_t nt = (count + kTile - 1) / kTile;  // <= kTile by construction
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t i = t * kTile + 4 * (int64_t)threadIdx.x;
    double q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = i + k < count ? __ldcg(v + i + k) : 0.0;
    const double s = block_tree_sum((q[0] + q[1]) + (q[2] + q[3]), scratch);
    if (threadIdx.x == 0) tile_sums[t] = s;
  }
  __syncthreads();
  return tile_sum4(tile_sums, 0, nt, scratch);
}

// Exclusive scan of in[0..count) (int) into out (long long) by one block of
// any multiple of 32 threads; returns the total.
__device__ long long block_exclusive_scan_any(const int* in, long long* out, int64_t count,
                                              long long* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nw = blockDim.x >> 5;
  long long carry = 0;
  for (int64_t base = 0; base < count; base += blockDim.x) {
    const int64_t i = base + tid;
    const long long v = i < count ? (long long)__ldcg(in + i) : 0;
    long long x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long w = lane < nw ? wsum[lane] : 0;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += y;
      }
      if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    const long long before = (warp > 0 ? wsum[warp - 1] : 0) + (x - v);
    if (i < count) out[i] = carry + before;
    const long long tot = wsum[nw - 1];
    __syncthreads();
    carry += tot;
  }
  return carry;
}

// 4 consecutive doubles v[i .. i + 3] (0 past n): two 16-byte vector loads
// when all four exist and v + i is 16-byte aligned (caller arrays of the
// step-level calls need only be 8-byte aligned), scalar loads otherwise.
__device__ __forceinline__ void load4(const double* v, int64_t i, int64_t n, double q[4]) {
  if (i + 3 < n && (reinterpret_cast<uintptr_t>(v + i) & 15u) == 0) {
    const double2 x = *reinterpret_cast<const double2*>(v + i);
    const double2 y = *reinterpret_cast<const double2*>(v + i + 2);
    q[0] = x.x;
    q[1] = x.y;
    q[2] = y.x;
    q[3] = y.y;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = i + k < n ? v[i + k] : 0.0;
  }
}

}  // namespace

__global__ void __launch_bounds__(kQuad) k_sum_status(const SweepArgs S) {
  __shared__ double scratch[33];
  __shared__ double tile_sums[kTile];
  __shared__ int is_last;
  if (S.st->flags & kDone) return;
  // a tile of kTile regions per block, 4 consecutive regions per thread
  const int64_t r = (int64_t)blockIdx.x * kTile + 4 * (int64_t)threadIdx.x;
  double a[4], b[4];
  load4(S.i7, r, S.n, a);
  load4(S.err, r, S.n, b);
  const double ta = block_tree_sum((a[0] + a[1]) + (a[2] + a[3]), scratch);
  const double tb = block_tree_sum((b[0] + b[1]) + (b[2] + b[3]), scratch);
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
  const double A = tree_sum_global4(S.blk_a, gridDim.x, scratch, tile_sums);
  const double B = tree_sum_global4(S.blk_b, gridDim.x, scratch, tile_sums);
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

__global__ void __launch_bounds__(kQuad) k_classify(const SweepArgs S) {
  __shared__ double scratch[33];
  __shared__ double tile_sums[kTile];
  __shared__ long long wsum[32];
  __shared__ int wcnt[kQuad / 32];
  __shared__ int is_last;
  if (S.st->flags & kDone) return;
  // a tile of kTile regions per block, 4 consecutive regions per thread
  const int64_t r = (int64_t)blockIdx.x * kTile + 4 * (int64_t)threadIdx.x;
  const double budget = S.budget_ptr ? *S.budget_ptr : S.budget_val;
  double i7[4], e[4], vf[4] = {0.0, 0.0, 0.0, 0.0};
  load4(S.i7, r, S.n, i7);
  load4(S.err, r, S.n, e);
  if (S.classifier != GMQ_LOCAL_REL) load4(S.volfrac, r, S.n, vf);
  uint8_t ax[4] = {0, 0, 0, 0};
  if (r + 3 < S.n && (reinterpret_cast<uintptr_t>(S.axis + r) & 3u) == 0) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(S.axis + r);
#pragma unroll
    for (int k = 0; k < 4; ++k) ax[k] = (uint8_t)(w >> (8 * k));
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) ax[k] = r + k < S.n ? S.axis[r + k] : 0;
  }
  int split = 0;
  double ri[4], re[4];
  uint8_t fl[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ri[k] = 0.0;
    re[k] = 0.0;
    fl[k] = 0;
    if (r + k < S.n) {
      const double thr = (S.classifier == GMQ_LOCAL_REL) ? __dmul_rn(S.rel_tol, fabs(i7[k]))
                                                         : __dmul_rn(budget, vf[k]);
      const double guard = __dmul_rn(S.guard, fabs(i7[k]));
      const bool retire = (e[k] <= thr) || (e[k] <= guard) || (ax[k] & 0x80);
      fl[k] = retire ? 0 : 1;
      split += fl[k];
      if (retire) {
        ri[k] = i7[k];
        re[k] = e[k];
      }
    }
  }
  if (r + 3 < S.n && (reinterpret_cast<uintptr_t>(S.flags + r) & 3u) == 0) {
    *reinterpret_cast<uint32_t*>(S.flags + r) =
        (uint32_t)fl[0] | ((uint32_t)fl[1] << 8) | ((uint32_t)fl[2] << 16) | ((uint32_t)fl[3] << 24);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (r + k < S.n) S.flags[r + k] = fl[k];
  }
  const int wsplit = __reduce_add_sync(0xffffffffu, split);
  if ((threadIdx.x & 31) == 0) wcnt[threadIdx.x >> 5] = wsplit;
  const double ta = block_tree_sum((ri[0] + ri[1]) + (ri[2] + ri[3]), scratch);  // syncs
  const double tb = block_tree_sum((re[0] + re[1]) + (re[2] + re[3]), scratch);
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int w = 0; w < kQuad / 32; ++w) cnt += wcnt[w];
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
  const long long total = block_exclusive_scan_any(S.blk_count, S.blk_off, gridDim.x, wsum);
  const double A = tree_sum_global4(S.blk_a, gridDim.x, scratch, tile_sums);
  const double B = tree_sum_global4(S.blk_b, gridDim.x, scratch, tile_sums);
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
  // four axes per step, every load issued before the stores
  for (int k0 = 0; k0 < S.d; k0 += 4) {
    double cv[4], hv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (k0 + q < S.d) {
        cv[q] = S.c[(int64_t)(k0 + q) * S.ld + r];
        hv[q] = S.h[(int64_t)(k0 + q) * S.ld + r];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q;
      if (k < S.d) {
        double cl = cv[q], cr = cv[q], hc = hv[q];
        if (k == ax) {
          hc = __dmul_rn(0.5, hv[q]);
          cl = __dsub_rn(cv[q], hc);
          cr = __dadd_rn(cv[q], hc);
        }
        S.c_out[(int64_t)k * S.ld_out + pos] = cl;
        S.h_out[(int64_t)k * S.ld_out + pos] = hc;
        S.c_out[(int64_t)k * S.ld_out + ns + pos] = cr;
        S.h_out[(int64_t)k * S.ld_out + ns + pos] = hc;
      }
    }
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
  k_sum_status<<<(unsigned)blocks, kQuad, 0, s>>>(S);
  return cudaGetLastError();
}

cudaError_t launch_classify(const SweepArgs& S, cudaStream_t s) {
  const int64_t blocks = (S.n + kTile - 1) / kTile;
  if (blocks == 0) return cudaSuccess;
  k_classify<<<(unsigned)blocks, kQuad, 0, s>>>(S);
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
