// gm_batch.cu -- many independent integrals in one device-resident loop
// (gmq_integrate_batch).  No counterpart in the paper, which integrates one
// problem at a time; every integral follows the paper's loop (Sec. 3, Fig.
// 1a) exactly as gmq_integrate runs it, but all of them advance together,
// one sweep per iteration, inside one CUDA graph.
//
// Layout: one region pool holds every integral's active regions; integral i
// owns the contiguous segment [off_i, off_i + n_i) of the current list (SoA,
// dmax rows, plus an int32 owner id per region).  Per sweep:
//   k_batch_rule64    one launch per family present (gm_batch_rule64.cuh):
//                     that family's regions, persistent grid, dimension per
//                     region; 1, 4, 32 or 128 lanes per region, chosen per
//                     sweep from the list length (the per-region work is
//                     gm_region64.cuh's, so the choice never changes a
//                     result); the mixed form's k_batch_rule_mixed likewise
//   k_batch_sums      tiles of 4096 regions of one integral each
//                     (persistent grid): pairwise-tree sums per tile; the
//                     integral's last tile adds the tile sums and tests the
//                     tolerance / sweep limit
//   k_batch_classify  per tile: flags, split count, retired pairwise-tree
//                     sums, round-off guard; the last tile: per-integral
//                     totals, first child position of every tile, cap
//   k_batch_scan      one block: new segment offsets (exclusive scan of
//                     2 n_split over the integrals still running), pool
//                     check, the next list's tile table
//   k_batch_split     per tile: left children then right children of its
//                     split regions into the integral's new segment
//   k_batch_restart   initial partitions of evicted integrals let in again
//   k_batch_commit    one thread per integral: its next segment
//   k_batch_advance   one thread: swap the lists, count the sweep, and set
//                     the graph's loop condition (bounded by max_iters)
// Per-integral sums use the same pairwise tree over the segment as the
// single-integral path, and the same child order, so every integral's
// result is the result gmq_integrate gives for it alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gm_batch.cuh"
#include "gm_region64.cuh"

namespace gmq {

namespace {

// Pairwise-tree sum of a tile of 4 * blockDim values, 4 consecutive values
// per thread: ((v0 + v1) + (v2 + v3)) is the first two levels of the tree.
__device__ __forceinline__ double tile_tree(double v0, double v1, double v2, double v3,
                                            double* scratch) {
  return block_tree_sum((v0 + v1) + (v2 + v3), scratch);
}

// The upper levels of an integral's pairwise tree: its tiles' sums ts[0 ..
// count), in groups of kSegBlock (complete subtrees), then the group sums
// (at most kSegBlock: segments up to 2^32 regions).  The partials were
// written by other blocks of this launch: read through L2 (__ldcg).
__device__ double tiles_tree_sum(const double* ts, long long count, double* scratch,
                                 double* gsum) {
  const int tid = threadIdx.x;
  const long long ngroups = (count + kSegBlock - 1) / kSegBlock;
  for (long long gi = 0; gi < ngroups; ++gi) {
    const long long t = gi * kSegBlock + tid;
    const double g = block_tree_sum(t < count ? __ldcg(ts + t) : 0.0, scratch);
    if (tid == 0) gsum[gi] = g;
  }
  __syncthreads();
  return block_tree_sum(tid < ngroups ? gsum[tid] : 0.0, scratch);
}

// The integral owning tile t: toff[i] <= t < toff[i + 1] (toff nondecreasing,
// toff[0] = 0 <= t < toff[count]).
__device__ __forceinline__ int tile_owner(const long long* toff, int count, long long t) {
  int lo = 0, hi = count;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (toff[mid] <= t)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Inclusive scan of one value per thread over a block of kSegBlock threads;
// *tot receives the block total.
__device__ long long block_incl_scan(long long v, long long* wsum, long long* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const long long incl = x + (warp > 0 ? wsum[warp - 1] : 0);
  *tot = wsum[31];
  __syncthreads();
  return incl;
}

}  // namespace

// ---------------------------------------------------------------------------

__global__ void k_batch_partition(const BatchArgs B) {
  const int id = blockIdx.x;
  const BatchItem& it = B.items[id];
  const int d = it.P.d;
  double* c = B.c[0];
  double* h = B.h[0];
  for (long long q = threadIdx.x; q < it.n; q += blockDim.x) {
    long long rem = q;
    const long long r = it.off + q;
    for (int k = 0; k < d; ++k) {
      const long long i = rem % it.s;
      rem /= it.s;
      c[(int64_t)k * B.ld + r] = __dadd_rn(it.lo[k], __dmul_rn((double)(2 * i + 1), it.h0[k]));
      h[(int64_t)k * B.ld + r] = it.h0[k];
    }
    B.rid[0][r] = id;
  }
}

// Global sums and convergence test of every integral (persistent grid over
// the current list's tiles): each tile's pairwise-tree sums of I7 and eps;
// the last of an integral's tiles to finish (ticket) adds the tile sums
// with the upper levels of the same tree and tests the tolerance.
__global__ void __launch_bounds__(kSegBlock) k_batch_sums(const BatchArgs B) {
  __shared__ double scratch[33];
  __shared__ double gsum[kSegBlock];
  __shared__ int owner, last;
  const long long* toff = B.tile_off[B.bs->parity];
  const long long nt = B.bs->n_tiles;
  for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
    if (threadIdx.x == 0) owner = tile_owner(toff, B.count, t);
    __syncthreads();
    BatchItem& it = B.items[owner];
    const long long t0 = toff[owner], ntl = toff[owner + 1] - t0;
    const long long base = (t - t0) * kSegTile;
    const long long cnt = it.n - base < kSegTile ? it.n - base : kSegTile;
    const int cur = B.bs->parity;
    const double* I7 = B.i7[cur] + it.off + base;
    const double* ER = B.err[cur] + it.off + base;
    const long long j = 4LL * threadIdx.x;
    const double a = tile_tree(j < cnt ? I7[j] : 0.0, j + 1 < cnt ? I7[j + 1] : 0.0,
                               j + 2 < cnt ? I7[j + 2] : 0.0, j + 3 < cnt ? I7[j + 3] : 0.0,
                               scratch);
    const double e = tile_tree(j < cnt ? ER[j] : 0.0, j + 1 < cnt ? ER[j + 1] : 0.0,
                               j + 2 < cnt ? ER[j + 2] : 0.0, j + 3 < cnt ? ER[j + 3] : 0.0,
                               scratch);
    if (threadIdx.x == 0) {
      B.tile_a[t] = a;
      B.tile_b[t] = e;
      __threadfence();
      last = atomicAdd(&it.tk_sum, 1u) == (unsigned)(ntl - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const double A = tiles_tree_sum(B.tile_a + t0, ntl, scratch, gsum);
      const double E2 = tiles_tree_sum(B.tile_b + t0, ntl, scratch, gsum);
      if (threadIdx.x == 0) {
        it.tk_sum = 0u;
        const double I = __dadd_rn(it.I_ret, A);
        const double E = __dadd_rn(it.E_ret, E2);
        const double budget = fmax(it.abs_tol, __dmul_rn(it.rel_tol, fabs(I)));
        it.I = I;
        it.E = E;
        it.budget = budget;
        it.iters += 1;
        it.regions += it.n;
        int f = it.flags;
        if (!isfinite(I) || !isfinite(E))
          f |= kNonfinite | kDone;
        else if (E <= budget)
          f |= kConverged | kDone;
        else if (it.iters >= B.bs->max_iters)
          f |= kLastSweep | kDone;
        it.flags = f;
      }
    }
    __syncthreads();
  }
}

// Classification of every integral's regions (persistent grid over tiles):
// flags, the tile's split count and its pairwise-tree sums of the retired
// regions; the last tile of an integral adds them up (retired sums with the
// upper tree levels), scans the tile counts into the tiles' first child
// positions, and applies the per-integral cap.
__global__ void __launch_bounds__(kSegBlock) k_batch_classify(const BatchArgs B) {
  __shared__ double scratch[33];
  __shared__ double gsum[kSegBlock];
  __shared__ long long wsum[32];
  __shared__ int owner, last, skip, cnt_s;
  const int cur = B.bs->parity;
  const long long* toff = B.tile_off[cur];
  const long long nt = B.bs->n_tiles;
  for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
    __syncthreads();  // every thread is done with the previous tile's shared values
    if (threadIdx.x == 0) {
      owner = tile_owner(toff, B.count, t);
      skip = (B.items[owner].flags & kDone) ? 1 : 0;
      cnt_s = 0;
    }
    __syncthreads();
    if (skip) continue;  // block-uniform; the integral stopped at the sums
    BatchItem& it = B.items[owner];
    const long long t0 = toff[owner], ntl = toff[owner + 1] - t0;
    const long long base = (t - t0) * kSegTile;
    const long long cnt = it.n - base < kSegTile ? it.n - base : kSegTile;
    const long long r0 = it.off + base;
    const double budget = it.budget;
    double ri[4], re[4];
    int c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long j = 4LL * threadIdx.x + q;
      ri[q] = 0.0;
      re[q] = 0.0;
      if (j < cnt) {
        const long long r = r0 + j;
        const double i7 = B.i7[cur][r], e = B.err[cur][r];
        const double thr = (B.classifier == GMQ_LOCAL_REL) ? __dmul_rn(it.rel_tol, fabs(i7))
                                                           : __dmul_rn(budget, B.vf[cur][r]);
        const bool retire =
            (e <= thr) || (e <= __dmul_rn(B.guard, fabs(i7))) || (B.axis[cur][r] & 0x80);
        B.flags[r] = retire ? 0 : 1;
        if (retire) {
          ri[q] = i7;
          re[q] = e;
        } else {
          ++c;
        }
      }
    }
    if (c) atomicAdd(&cnt_s, c);
    const double a = tile_tree(ri[0], ri[1], ri[2], ri[3], scratch);  // syncs: cnt_s is final
    const double e = tile_tree(re[0], re[1], re[2], re[3], scratch);
    if (threadIdx.x == 0) {
      B.tile_cnt[t] = cnt_s;
      B.tile_a[t] = a;
      B.tile_b[t] = e;
      __threadfence();
      last = atomicAdd(&it.tk_cls, 1u) == (unsigned)(ntl - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      // split count and the tiles' first child positions (exclusive scan)
      long long carry = 0, tot = 0;
      for (long long b0 = 0; b0 < ntl; b0 += kSegBlock) {
        const long long q = b0 + threadIdx.x;
        const long long v = q < ntl ? __ldcg(B.tile_cnt + t0 + q) : 0;
        const long long incl = block_incl_scan(v, wsum, &tot);
        if (q < ntl) B.tile_pos[t0 + q] = carry + incl - v;
        carry += tot;
      }
      const double rsum = tiles_tree_sum(B.tile_a + t0, ntl, scratch, gsum);
      const double esum = tiles_tree_sum(B.tile_b + t0, ntl, scratch, gsum);
      if (threadIdx.x == 0) {
        it.tk_cls = 0u;
        const long long total = carry;
        it.n_split = total;
        int f = it.flags;
        if (total == 0 || 2 * total > it.cap) {
          // the integral stops this sweep either way: commit now
          it.I_ret = __dadd_rn(it.I_ret, rsum);
          it.E_ret = __dadd_rn(it.E_ret, esum);
          f |= (total == 0 ? kAllRetired : kCapExceeded) | kDone;
        } else {
          // committed by the scan if the split fits in the pool this sweep
          it.ret_i = rsum;
          it.ret_e = esum;
        }
        it.flags = f;
      }
    }
    __syncthreads();
  }
}

// Pool allocation of the next list.  Every running integral first keeps
// room for its current regions (their total fits: they are in the pool
// now); integrals whose list shrinks always split; the growing ones split
// while the running sum of their growth, in index order, fits in the rest
// of the pool.  A growing integral that does not fit is paused: it keeps
// this sweep's regions unchanged, its retired sums are not committed and
// its counters are rolled back, so next sweep it re-evaluates the same
// regions and takes the same decisions (its result is unchanged, only
// later).  If nothing can split while some integral is paused, the paused
// integral with the highest index is evicted: its regions and state are
// dropped and it waits, holding nothing, until the pool has room for its
// initial partition, when it starts over (deterministically, so again with
// its single-run result).  Evicted integrals restart in index order.  An
// integral that cannot grow even with the pool to itself stops (cap).
__global__ void __launch_bounds__(kSegBlock) k_batch_scan(const BatchArgs B) {
  __shared__ long long wsum[32];
  __shared__ int active_s, admitted_s, paused_hi, paused_lo, running_s, stop_first;
  const int tid = threadIdx.x;
  if (tid == 0) {
    active_s = 0;
    admitted_s = 0;
    paused_hi = -1;
    paused_lo = 0x7fffffff;
    running_s = 0;
    stop_first = 0;
  }
  __syncthreads();
  auto running = [&](int i) {
    return i < B.count && !(B.items[i].flags & kDone) && !B.items[i].deferred;
  };
  long long tot = 0, R = 0;
  for (int base = 0; base < B.count; base += kSegBlock) {
    const int i = base + tid;
    const bool run = running(i);
    if (run) atomicAdd(&running_s, 1);
    block_incl_scan(run ? B.items[i].n : 0, wsum, &tot);
    R += tot;
  }
  const long long budget = B.pool_cap - R;
  long long carry = 0;
  for (int base = 0; base < B.count; base += kSegBlock) {
    const int i = base + tid;
    const bool run = running(i);
    long long grow = 0;
    if (run) grow = 2 * B.items[i].n_split - B.items[i].n;
    const long long pre = carry + block_incl_scan(grow > 0 ? grow : 0, wsum, &tot);
    if (run) {
      const bool admit = grow <= 0 || pre <= budget;
      B.items[i].paused = admit ? 0 : 1;
      if (admit) {
        atomicOr(&admitted_s, 1);
      } else {
        atomicMax(&paused_hi, i);
        atomicMin(&paused_lo, i);
      }
    }
    carry += tot;
  }
  __syncthreads();
  // Nothing can split: make room for the paused integral of lowest index
  // (f) by evicting paused integrals from the highest index down, as few as
  // free its missing room; if evicting all of them would not be enough, f
  // cannot grow in this pool and stops instead.  Evicted integrals drop
  // their regions and state and restart later from their initial partition.
  if (admitted_s == 0 && paused_hi >= 0) {
    const int f = paused_lo;
    const long long need = (2 * B.items[f].n_split - B.items[f].n) - budget;
    long long carry2 = 0, all = 0;
    for (int base = 0; base < B.count; base += kSegBlock) {  // total of the others
      const int i = base + tid;
      const bool cand = i < B.count && i != f && running(i) && B.items[i].paused;
      block_incl_scan(cand ? B.items[i].n : 0, wsum, &tot);
      all += tot;
    }
    if (all < need) {
      if (tid == 0) stop_first = 1;
    } else {
      for (int base = 0; base < B.count; base += kSegBlock) {  // suffix sums, high index first
        const int i = B.count - 1 - (base + tid);
        const bool cand = i >= 0 && i != f && running(i) && B.items[i].paused;
        const long long suffix = carry2 + block_incl_scan(cand ? B.items[i].n : 0, wsum, &tot);
        if (cand && suffix - B.items[i].n < need) {
          BatchItem& v = B.items[i];
          v.paused = 0;
          v.deferred = 2;  // evicted this sweep: not restarted before the next
          v.I_ret = v.E_ret = 0.0;
          v.iters = 0;
          v.regions = 0;
          v.n = 0;
          atomicAdd(&B.bs->evictions, 1);
        }
        carry2 += tot;
      }
    }
    __syncthreads();
    if (tid == 0 && stop_first) {
      BatchItem& v = B.items[f];
      v.paused = 0;
      v.flags |= kCapExceeded | kDone;
    }
  }
  __syncthreads();
  // sizes of the next list for the running integrals
  long long used = 0;
  for (int base = 0; base < B.count; base += kSegBlock) {
    const int i = base + tid;
    long long size = 0;
    if (running(i)) {
      BatchItem& it = B.items[i];
      size = it.paused ? it.n : 2 * it.n_split;
    }
    block_incl_scan(size, wsum, &tot);
    used += tot;
  }
  // waiting integrals (evicted, or not yet admitted) start, in index order,
  // only in a sweep where nothing had to pause, and only while their
  // initial partitions leave a quarter of the pool free for growth: an
  // integral started into a full pool would only be evicted again
  const bool slack = paused_hi < 0;
  const long long room = B.pool_cap - used - B.pool_cap / 4;
  carry = 0;
  for (int base = 0; base < B.count; base += kSegBlock) {
    const int i = base + tid;
    const bool waiting = i < B.count && !(B.items[i].flags & kDone) && B.items[i].deferred == 1;
    const long long need = waiting ? B.items[i].n0 : 0;
    const long long pre = carry + block_incl_scan(need, wsum, &tot);
    if (waiting && slack && pre <= room) {
      B.items[i].deferred = 0;
      B.items[i].restart = 1;
    }
    carry += tot;
  }
  __syncthreads();
  carry = 0;
  long long* toff_next = B.tile_off[B.bs->parity ^ 1];
  long long ttot = 0, tcarry = 0;
  for (int base = 0; base < B.count; base += kSegBlock) {
    const int i = base + tid;
    long long size = 0;
    if (i < B.count) {
      BatchItem& it = B.items[i];
      if (!(it.flags & kDone)) {
        if (it.restart) {
          size = it.n0;
        } else if (it.deferred) {
          size = 0;
          it.deferred = 1;
        } else if (it.paused) {
          size = it.n;
          it.iters -= 1;
          it.regions -= it.n;
          atomicAdd(&B.bs->pauses, 1);
          atomicAdd(reinterpret_cast<unsigned long long*>(&B.bs->carried_next),
                    (unsigned long long)it.n);
        } else {
          size = 2 * it.n_split;
          it.I_ret = __dadd_rn(it.I_ret, it.ret_i);
          it.E_ret = __dadd_rn(it.E_ret, it.ret_e);
        }
        atomicAdd(&active_s, 1);
      }
    }
    const long long incl = block_incl_scan(size, wsum, &tot);
    if (i < B.count) {
      B.items[i].noff = carry + incl - size;
      B.items[i].nnext = size;
      for (int f = 0; f < 7; ++f)
        if (i == B.fam_item_lo[f]) B.bs->fam_off[B.bs->parity ^ 1][f] = carry + incl - size;
    }
    carry += tot;
    // tiles of the next list
    const long long tiles = (size + kSegTile - 1) / kSegTile;
    const long long tincl = block_incl_scan(tiles, wsum, &ttot);
    if (i < B.count) toff_next[i] = tcarry + tincl - tiles;
    tcarry += ttot;
  }
  __syncthreads();
  if (tid == 0) {
    B.bs->n_next = carry;
    B.bs->active = active_s;
    B.bs->n_tiles_next = tcarry;
    toff_next[B.count] = tcarry;
    for (int f = 0; f < 8; ++f)
      if (B.fam_item_lo[f] >= B.count) B.bs->fam_off[B.bs->parity ^ 1][f] = carry;
  }
}

// Bisection (persistent grid over the current list's tiles): the split
// regions of a tile go, in order, to positions tile_pos[t] + (split regions
// before them in the tile) of their integral's new segment -- left children
// first, right children n_split positions later; a paused integral's tile
// is copied unchanged.
__global__ void __launch_bounds__(kSegBlock) k_batch_split(const BatchArgs B) {
  __shared__ int wcount[32];
  __shared__ int owner, skip;
  const int cur = B.bs->parity, nxt = cur ^ 1;
  const long long* toff = B.tile_off[cur];
  const long long nt = B.bs->n_tiles;
  const double* C = B.c[cur];
  const double* H = B.h[cur];
  double* Co = B.c[nxt];
  double* Ho = B.h[nxt];
  int32_t* rido = B.rid[nxt];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
    __syncthreads();
    if (tid == 0) {
      owner = tile_owner(toff, B.count, t);
      const BatchItem& w = B.items[owner];
      skip = ((w.flags & kDone) || w.deferred) ? 1 : 0;
    }
    __syncthreads();
    if (skip) continue;
    const int id = owner;
    const BatchItem& it = B.items[id];
    const long long t0 = toff[id];
    const long long base = (t - t0) * kSegTile;
    const long long cnt = it.n - base < kSegTile ? it.n - base : kSegTile;
    const long long r0 = it.off + base, noff = it.noff, ns = it.n_split;
    const int d = it.P.d;
    if (it.paused) {
      // no room this sweep: carry the tile over unchanged, with its rule
      // outputs (the next sweep does not evaluate it again)
      for (long long j = tid; j < cnt; j += kSegBlock) {
        const long long q = noff + base + j, r = r0 + j;
        for (int k = 0; k < d; ++k) {
          Co[(int64_t)k * B.ld + q] = C[(int64_t)k * B.ld + r];
          Ho[(int64_t)k * B.ld + q] = H[(int64_t)k * B.ld + r];
        }
        rido[q] = (int32_t)id;
        B.i7[nxt][q] = B.i7[cur][r];
        B.err[nxt][q] = B.err[cur][r];
        B.vf[nxt][q] = B.vf[cur][r];
        B.axis[nxt][q] = B.axis[cur][r];
      }
      continue;
    }
    long long carry = B.tile_pos[t];
    for (long long b0 = 0; b0 < cnt; b0 += kSegBlock) {
      const long long j = b0 + tid;
      const long long r = r0 + j;
      const int f = (j < cnt) ? (int)B.flags[r] : 0;
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (lane == 0) wcount[warp] = __popc(bal);
      __syncthreads();
      int wpre = 0, tot = 0;
      for (int w = 0; w < kSegBlock / 32; ++w) {
        if (w < warp) wpre += wcount[w];
        tot += wcount[w];
      }
      if (f) {
        const long long pos = carry + wpre + __popc(bal & ((1u << lane) - 1u));
        const int ax = B.axis[cur][r] & 0x7f;
        for (int k = 0; k < d; ++k) {
          const double cv = C[(int64_t)k * B.ld + r];
          const double hv = H[(int64_t)k * B.ld + r];
          double cl = cv, cr = cv, hc = hv;
          if (k == ax) {
            hc = __dmul_rn(0.5, hv);
            cl = __dsub_rn(cv, hc);
            cr = __dadd_rn(cv, hc);
          }
          Co[(int64_t)k * B.ld + noff + pos] = cl;
          Ho[(int64_t)k * B.ld + noff + pos] = hc;
          Co[(int64_t)k * B.ld + noff + ns + pos] = cr;
          Ho[(int64_t)k * B.ld + noff + ns + pos] = hc;
        }
        rido[noff + pos] = (int32_t)id;
        rido[noff + ns + pos] = (int32_t)id;
      }
      carry += tot;
      __syncthreads();  // wcount is rewritten by the next chunk
    }
  }
}

// An evicted integral the scan let in again starts over: its initial
// partition at its new offset (one block per integral; others return).
__global__ void k_batch_restart(const BatchArgs B) {
  const BatchItem& it = B.items[blockIdx.x];
  if (!it.restart || (it.flags & kDone)) return;
  const int nxt = B.bs->parity ^ 1;
  const int d = it.P.d;
  for (long long q = threadIdx.x; q < it.n0; q += blockDim.x) {
    long long rem = q;
    for (int k = 0; k < d; ++k) {
      const long long i = rem % it.s;
      rem /= it.s;
      B.c[nxt][(int64_t)k * B.ld + it.noff + q] =
          __dadd_rn(it.lo[k], __dmul_rn((double)(2 * i + 1), it.h0[k]));
      B.h[nxt][(int64_t)k * B.ld + it.noff + q] = it.h0[k];
    }
    B.rid[nxt][it.noff + q] = (int32_t)blockIdx.x;
  }
}

// Every running integral's segment in the next list (one thread each).
__global__ void k_batch_commit(const BatchArgs B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B.count) return;
  BatchItem& it = B.items[i];
  if ((it.flags & kDone) || it.deferred) return;
  it.off = it.noff;
  it.n = it.nnext;
  it.restart = 0;
}

// Copies of the initial list's regions [0, n0) into [n0, n), cyclically
// (the autotuner's larger lists; valid regions of real integrals).
__global__ void k_batch_tile(const BatchArgs B, long long n0, long long n) {
  const long long i = n0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long src = i % n0;
  for (int k = 0; k < B.dmax; ++k) {
    B.c[0][(int64_t)k * B.ld + i] = B.c[0][(int64_t)k * B.ld + src];
    B.h[0][(int64_t)k * B.ld + i] = B.h[0][(int64_t)k * B.ld + src];
  }
  B.rid[0][i] = B.rid[0][src];
}

__global__ void k_batch_advance(const BatchArgs B) {
  BatchState* bs = B.bs;
  const int used = bs->lanes;
  bs->lane_sweeps[used == 128 ? 3 : (used == 32 ? 2 : (used == 4 ? 1 : 0))] += 1;
  // the current list's regions were evaluated unless carried over
  bs->list_regions += bs->n_total;
  bs->rule_regions += bs->n_total - bs->carried_cur;
  bs->carried_regions += bs->carried_next;
  bs->carried_cur = bs->carried_next;
  bs->carried_next = 0;
  bs->n_total = bs->n_next;
  bs->n_tiles = bs->n_tiles_next;
  bs->parity ^= 1;
  bs->sweep += 1;
  bs->lanes = batch_lanes_for(B, bs->n_total);
  // problems waiting for room count as active: a sweep with no regions
  // still runs the scan that starts them
  const bool more = bs->active > 0 && bs->sweep < bs->max_sweeps;
  if (B.use_cond) cudaGraphSetConditional(B.cond, more ? 1u : 0u);
}

size_t batch_rule_smem(int dmax) {
  const size_t pairs = sizeof(unsigned short) * (size_t)batch_pairs_offset(dmax + 1);
  return (sizeof(double) * (size_t)batch_rule_doubles_max(dmax) + pairs + 15) & ~(size_t)15;
}

cudaError_t batch_launch_partition(const BatchArgs& B, cudaStream_t s) {
  k_batch_partition<<<B.count, 256, 0, s>>>(B);
  return cudaGetLastError();
}

cudaError_t batch_launch_tile(const BatchArgs& B, long long n0, long long n, cudaStream_t s) {
  if (n <= n0) return cudaSuccess;
  const long long blocks = (n - n0 + 255) / 256;
  k_batch_tile<<<(unsigned)blocks, 256, 0, s>>>(B, n0, n);
  return cudaGetLastError();
}

cudaError_t batch_launch_rest(const BatchArgs& B, cudaStream_t s) {
  k_batch_sums<<<B.tile_grid, kSegBlock, 0, s>>>(B);
  k_batch_classify<<<B.tile_grid, kSegBlock, 0, s>>>(B);
  k_batch_scan<<<1, kSegBlock, 0, s>>>(B);
  k_batch_split<<<B.tile_grid, kSegBlock, 0, s>>>(B);
  k_batch_restart<<<B.count, 256, 0, s>>>(B);
  k_batch_commit<<<(B.count + 255) / 256, 256, 0, s>>>(B);
  k_batch_advance<<<1, 1, 0, s>>>(B);
  return cudaGetLastError();
}

}  // namespace gmq
