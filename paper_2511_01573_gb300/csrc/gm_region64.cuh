// gm_region64.cuh -- FP64 evaluation of one region by a group of T lanes
// (T in {1, 4, 32, 128}: a thread, four lanes, a warp or a 128-thread block
// per region), shared by the single-integral rule kernel (gm_rule.cuh)
// and the batched rule kernel (gm_batch.cu): both compute every region with
// the same operations in the same order.
//
// What is computed (paper Sec. 2, the Genz-Malik degree-7 rule with its
// embedded degree-5 rule): the five class sums S1..S5 of f over the fully
// symmetric node classes, the fourth differences D_k from the centre and
// the +-lambda2, +-lambda3 axis nodes, and the split axis argmax_k D_k.
//
// Summation order.  Every class sum is one fixed tree, whatever T is.  The
// class's nodes, in the order of their definition (class 2: axis k = 0..d-1,
// +lambda2 then -lambda2; class 3 likewise with lambda3; class 4: pairs
// j < k in lexicographic order, sign patterns ++, +-, -+, --; class 5: sign
// patterns m = 0 .. 2^d - 1, bit j set = -lambda5 on axis j) are cut into
// 128 chunks of c = ceil(n / 128) consecutive nodes (trailing chunks may be
// short or empty).  A chunk is summed left to right; the chunk sums are
// combined by the adjacent-pairwise tree over the 128 chunk positions, in
// which a subtree holding no node passes its sibling through unchanged.
// Lane l of a group of T takes the 128/T consecutive chunks that start at
// chunk (128/T) * bitrev(l) (bitrev over log2 T bits), combines them with
// the same tree, and the group finishes the tree with an xor butterfly:
// with that bit-reversed assignment the butterfly's partners at offset T/2,
// T/4, ... are exactly the tree's sibling subtrees at successive levels, and
// IEEE addition is commutative, so every lane ends with the same value.  The
// sums -- and everything computed from them -- are therefore bit-identical
// for T = 1, 4, 32 and 128: the lane mapping is a pure launch choice.
#pragma once

#include "gmq_common.cuh"
#include "gmq_families.cuh"

namespace gmq {

// Node-coordinate rows of a region's table (lambda4 == lambda3, so pair
// nodes reuse rows P3/M3).
enum XRow { kXC = 0, kXP2 = 1, kXM2 = 2, kXP3 = 3, kXM3 = 4, kXP5 = 5, kXM5 = 6, kXRows = 7 };

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }

// Chunks per class: the width of every class-sum tree, and the largest
// group of lanes per region (a 128-thread block).
constexpr int kChunks = 128;

// Lanes of this thread's group within its warp (T consecutive lanes of one
// warp; for T = 128 the group is the whole block and each warp takes part
// with all its lanes).
template <int T>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (T >= 32) {
    return 0xffffffffu;
  } else {
    const unsigned base = (threadIdx.x & 31u) & ~(unsigned)(T - 1);
    return ((1u << T) - 1u) << base;
  }
}

// Synchronise the lanes of a group (the block for T = 128).
template <int T>
__device__ __forceinline__ void group_sync(unsigned mask) {
  if constexpr (T > 32)
    __syncthreads();
  else
    __syncwarp(mask);
}

// First of the kChunks/T chunk positions lane `lane` of a group of T owns.
template <int T>
__device__ __forceinline__ int lane_first_chunk(int lane) {
  if constexpr (T == 1) {
    return 0;
  } else {
    constexpr int bits = ilog2c(T);
    return (kChunks / T) * (int)(__brev((unsigned)lane) >> (32 - bits));
  }
}

// Adjacent-pairwise tree over at most 128 leaves pushed left to right: a
// binary counter of complete subtrees (L[j] holds 2^j leaves while bit j of
// the leaf count is set).  flush() combines the pending subtrees from the
// rightmost up, so a missing right part of the tree passes through.
struct PairTree {
  double L0 = 0.0, L1 = 0.0, L2 = 0.0, L3 = 0.0, L4 = 0.0, L5 = 0.0, L6 = 0.0, L7 = 0.0;
  int n = 0;
  __device__ __forceinline__ void push(double x) {
    const int p = n++;
    if (!(p & 1)) { L0 = x; return; }
    x = __dadd_rn(L0, x);
    if (!(p & 2)) { L1 = x; return; }
    x = __dadd_rn(L1, x);
    if (!(p & 4)) { L2 = x; return; }
    x = __dadd_rn(L2, x);
    if (!(p & 8)) { L3 = x; return; }
    x = __dadd_rn(L3, x);
    if (!(p & 16)) { L4 = x; return; }
    x = __dadd_rn(L4, x);
    if (!(p & 32)) { L5 = x; return; }
    x = __dadd_rn(L5, x);
    if (!(p & 64)) { L6 = x; return; }
    L7 = __dadd_rn(L6, x);
  }
  __device__ __forceinline__ double flush(bool& present) const {
    present = n > 0;
    if (n >= 128) return L7;
    double x = 0.0;
    bool have = false;
    if (n & 1) { x = L0; have = true; }
    if (n & 2) { x = have ? __dadd_rn(L1, x) : L1; have = true; }
    if (n & 4) { x = have ? __dadd_rn(L2, x) : L2; have = true; }
    if (n & 8) { x = have ? __dadd_rn(L3, x) : L3; have = true; }
    if (n & 16) { x = have ? __dadd_rn(L4, x) : L4; have = true; }
    if (n & 32) { x = have ? __dadd_rn(L5, x) : L5; have = true; }
    if (n & 64) { x = have ? __dadd_rn(L6, x) : L6; }
    return x;
  }
};

// Combine a lane's partial with its butterfly partner's (absent partials
// pass the other side through); a + b == b + a, so both partners agree.
__device__ __forceinline__ void tree_combine(double& x, bool& present, double ox, bool op) {
  if (present && op) {
    x = __dadd_rn(x, ox);
  } else if (op) {
    x = ox;
    present = true;
  }
}

// The group's xor butterfly over lane partial trees; every lane returns the
// full tree's value.  T = 128: the two levels across warps (offsets 64, 32)
// go through shared memory, the rest through warp shuffles.
template <int T>
__device__ __forceinline__ double lanes_tree(double x, bool present, unsigned mask) {
  if constexpr (T > 32) {
    __shared__ double sx[T];
    __shared__ int sp[T];
    const int l = threadIdx.x & (T - 1);
#pragma unroll
    for (int off = T / 2; off >= 32; off >>= 1) {
      __syncthreads();
      sx[l] = x;
      sp[l] = present ? 1 : 0;
      __syncthreads();
      tree_combine(x, present, sx[l ^ off], sp[l ^ off] != 0);
    }
  }
  constexpr int W = T < 32 ? T : 32;
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) {
    const double ox = __shfl_xor_sync(mask, x, off, W);
    const int op = __shfl_xor_sync(mask, present ? 1 : 0, off, W);
    tree_combine(x, present, ox, op != 0);
  }
  return present ? x : 0.0;
}

// One class sum over n nodes, val(q) = f at the class's node q.
template <int T, class Val>
__device__ __forceinline__ double class_sum(int n, int lane, unsigned mask, Val val) {
  PairTree t;
  if (n > 0) {
    const int c = (n + kChunks - 1) / kChunks;
    const int nch = (n + c - 1) / c;
    const int p0 = lane_first_chunk<T>(lane);
    const int p1 = min(p0 + kChunks / T, nch);
    for (int p = p0; p < p1; ++p) {
      const int q0 = p * c, q1 = min(q0 + c, n);
      // the chunk's first node starts the sum (no add of a zero: a select
      // would leave the add in the instruction stream)
      double x = val(q0);
      for (int q = q0 + 1; q < q1; ++q) x = __dadd_rn(x, val(q));
      t.push(x);
    }
  }
  bool present;
  const double x = t.flush(present);
  return lanes_tree<T>(x, present, mask);
}

struct RegionSums {
  double s1, s2, s3, s4, s5;  // class sums
  double f0;                  // f(centre)
  double dbest;               // largest fourth difference
  int kbest;                  // its axis (lowest on ties)
};

// Separable node sums.  Every family is f = g(S), S = base (+) phi_0(x_0)
// (+) ... (+) phi_{d-1}(x_{d-1}) (Sep<FAM> in gmq_families.cuh), and a
// node's coordinate on axis j is one of seven values: the centre c_j or
// c_j +- lambda h_j.  So a region evaluates phi 7 d times and forms each
// node's S from a fixed association of per-axis terms and partial chains:
//   pre_k = base (+) phi_C(0) (+) ... (+) phi_C(k-1)        (left to right)
//   suf_k = phi_C(k) (+) (phi_C(k+1) (+) (... phi_C(d-1)))  (right to left)
//   centre             S = base (+) suf_0
//   axis node (k, x)   S = (pre_k (+) phi_k(x)) (+) suf_{k+1}
//   pair node (j<k)    S = ((pre_j (+) phi_j(x_j)) (+) mid_jk) (+)
//                          (phi_k(x_k) (+) suf_{k+1}),
//                      mid_jk = phi_C(j+1) (+) ... (+) phi_C(k-1) (left to right)
//   class-5 node m     S = A[m_A] (+) (B[m_B] (+) C[m_C])
// where the sign pattern m is cut into parts over axes [0, a), [a, a + b),
// [a + b, d) and A, B, C hold the left-to-right chains over each part
// (base heading A).  An empty operand (no base, k = 0; k = d - 1; an empty
// middle or part) is left out rather than combined with an identity.  With
// one combine per node (two for the pair nodes' shared prefix, amortised
// over their four sign patterns) the per-node FP64 work is the outer
// function g and the accumulation.  S differs from the plain left-to-right
// chain only in rounding order; every lane mapping forms it the same way, so
// the class sums stay bit-identical for T = 1, 4, 32 and 128.

// Parts of the class-5 sign pattern: two for d <= 8, three above.
__host__ __device__ constexpr int sep_c(int d) { return d <= 8 ? 0 : d / 3; }
__host__ __device__ constexpr int sep_b(int d) { return d <= 8 ? d / 2 : (d - d / 3) / 2; }
__host__ __device__ constexpr int sep_a(int d) { return d - sep_b(d) - sep_c(d); }

// Workspace of one region (entries `stride` doubles apart): phi at the
// centre [d], the pair-node prefixes L[k][s] = pre_k (+) phi_k(c +- lambda3 h)
// [2d], the suffixes R[k][s] = phi_k(c +- lambda3 h) (+) suf_{k+1} [2d], the
// class-5 chains A [2^a], B [2^b or 0], C [2^c or 0], for the discontinuous
// family the flag masks [2]; with T > 1 lanes also pre_k [d], suf_{k+1} [d],
// the centre's S [1] and the axis-node values [4d + 1] the lanes share.
struct SepLayout {
  int phiC, L, R, A, B, C, Z, pre, suf, sc, fv, words;
};

__host__ __device__ constexpr SepLayout sep_layout(int d, bool flag, bool lanes) {
  SepLayout s{};
  s.phiC = 0;
  s.L = d;
  s.R = 3 * d;
  s.A = 5 * d;
  s.B = s.A + (1 << sep_a(d));
  s.C = s.B + (sep_b(d) ? 1 << sep_b(d) : 0);
  s.Z = s.C + (sep_c(d) ? 1 << sep_c(d) : 0);
  int w = s.Z + (flag ? 2 : 0);
  s.pre = s.suf = s.sc = s.fv = -1;
  if (lanes) {
    s.pre = w;
    s.suf = w + d;
    s.sc = w + 2 * d;
    s.fv = w + 2 * d + 1;
    w += 2 * d + 1 + 4 * d + 1;
  }
  s.words = w;
  return s;
}

// The largest workspace over dimensions 1 .. dmax (batched kernels, whose
// regions have different dimensions).
__host__ __device__ constexpr int sep_words_max(int dmax, bool flag, bool lanes) {
  int m = 0;
  for (int d = 1; d <= dmax; ++d)
    if (sep_layout(d, flag, lanes).words > m) m = sep_layout(d, flag, lanes).words;
  return m;
}

// The class sums and the fourth-difference argmax of one region by the T
// lanes of the calling group (all of them call it).  ch(k, c, h) loads the
// region's centre and half-width on axis k; pairs[p] = (j << 8) | k for the
// p-th pair j < k of dimension d; w points at the region's workspace
// (sep_layout(d, Sep<FAM>::kFlag, T > 1)), entries `ws` doubles apart.
template <int FAM, int T, class PT, class CH>
__device__ __forceinline__ void region_sums64(const PT& P, int d, const unsigned short* pairs,
                                              const CH& ch, double lam2, double lam3,
                                              double lam5, double* w, int ws, double ratio,
                                              RegionSums& o) {
  using SF = Sep<FAM>;
  const int lane = (T == 1) ? 0 : (int)(threadIdx.x & (unsigned)(T - 1));
  const unsigned mask = group_mask<T>();
  const SepLayout Ly = sep_layout(d, SF::kFlag, T > 1);
  const int pa = sep_a(d), pb = sep_b(d), pc = sep_c(d);
  auto W = [&](int e) -> double& { return w[(long long)e * ws]; };
  auto op = [](double x, double y) -> double {
    if constexpr (SF::kMul)
      return __dmul_rn(x, y);
    else
      return __dadd_rn(x, y);
  };
  auto fval = [&](double S, bool zero) -> double {
    if constexpr (SF::kFlag) {
      if (zero) return 0.0;
    }
    return SF::g(d, S);
  };
  // generator of axis-node row r: +lambda2, -lambda2, +lambda3, -lambda3
  auto lam_row = [&](int r) -> double {
    return r < 2 ? (r ? -lam2 : lam2) : (r == 2 ? lam3 : -lam3);
  };
  // discontinuous family: flag bits (x_j > u_j) of the centre, of
  // c +- lambda3 h (+ in bits 0..15, - in bits 16..31) and of c +- lambda5 h
  unsigned zc = 0u, z3 = 0u, z5 = 0u;
  double f0, s2, s3, dbest = -1.0;
  int kbest = 0;
  if constexpr (T == 1) {
    // right to left: phi at the centre, R, suf (suf_{k+1} parked in L[k][0],
    // phi at c +- lambda3 h parked in the class-5 chain area, which holds at
    // least 2d entries and is filled only after the axis nodes)
    double suf = 0.0;
    for (int k = d - 1; k >= 0; --k) {
      double c, h;
      ch(k, c, h);
      const double xp = fma(lam3, h, c), xm = fma(-lam3, h, c);
      const double fc = SF::phi(P, k, c), fp = SF::phi(P, k, xp), fm = SF::phi(P, k, xm);
      if constexpr (SF::kFlag) {
        zc |= (unsigned)SF::flag(P, k, c) << k;
        z3 |= ((unsigned)SF::flag(P, k, xp) << k) | ((unsigned)SF::flag(P, k, xm) << (k + 16));
      }
      W(Ly.phiC + k) = fc;
      W(Ly.A + 2 * k) = fp;
      W(Ly.A + 2 * k + 1) = fm;
      if (k == d - 1) {
        W(Ly.R + 2 * k) = fp;
        W(Ly.R + 2 * k + 1) = fm;
        suf = fc;
      } else {
        W(Ly.R + 2 * k) = op(fp, suf);
        W(Ly.R + 2 * k + 1) = op(fm, suf);
        W(Ly.L + 2 * k) = suf;
        suf = op(fc, suf);
      }
    }
    f0 = fval(SF::kBase ? op(SF::base(P), suf) : suf, zc != 0u);
    const double two_f0 = __dmul_rn(2.0, f0);
    // left to right: the axis nodes (classes 2 and 3 in their order, the
    // fourth differences) and the pair-node prefixes L
    PairTree t2, t3;
    double pre = SF::kBase ? SF::base(P) : 0.0;
    bool hp = SF::kBase;
    for (int k = 0; k < d; ++k) {
      double c, h;
      ch(k, c, h);
      const bool hs = k < d - 1;
      const double sk = hs ? W(Ly.L + 2 * k) : 0.0;
      double q[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        double ph;
        bool fx = false;
        if (r < 2) {
          const double x = fma(lam_row(r), h, c);
          ph = SF::phi(P, k, x);
          if constexpr (SF::kFlag) fx = SF::flag(P, k, x);
        } else {
          ph = W(Ly.A + 2 * k + (r - 2));  // parked by the first pass
          if constexpr (SF::kFlag) fx = (z3 >> (k + 16 * (r - 2))) & 1u;
        }
        const double lp = hp ? op(pre, ph) : ph;
        if (r >= 2) W(Ly.L + 2 * k + (r - 2)) = lp;  // after suf_{k+1} was read
        bool zero = false;
        if constexpr (SF::kFlag) zero = ((zc & ~(1u << k)) != 0u) || fx;
        q[r] = fval(hs ? op(lp, sk) : lp, zero);
      }
      t2.push(q[0]);
      t2.push(q[1]);
      t3.push(q[2]);
      t3.push(q[3]);
      const double t1 = __dsub_rn(__dadd_rn(q[0], q[1]), two_f0);
      const double tt = __dsub_rn(__dadd_rn(q[2], q[3]), two_f0);
      const double D = fabs(__dsub_rn(t1, __dmul_rn(ratio, tt)));
      if (D > dbest) {
        dbest = D;
        kbest = k;
      }
      const double fck = W(Ly.phiC + k);
      pre = hp ? op(pre, fck) : fck;
      hp = true;
    }
    bool pr;
    s2 = t2.flush(pr);
    s3 = t3.flush(pr);
    // class-5 chains, by doubling: after axis j0 + i the first 2^(i+1)
    // entries hold the chains over axes j0 .. j0 + i
    auto chains = [&](int e0, int j0, int nb, bool with_base) {
      for (int i = 0; i < nb; ++i) {
        double c, h;
        ch(j0 + i, c, h);
        const double xp = fma(lam5, h, c), xm = fma(-lam5, h, c);
        const double fp = SF::phi(P, j0 + i, xp), fm = SF::phi(P, j0 + i, xm);
        if constexpr (SF::kFlag)
          z5 |= ((unsigned)SF::flag(P, j0 + i, xp) << (j0 + i)) |
                ((unsigned)SF::flag(P, j0 + i, xm) << (j0 + i + 16));
        if (i == 0) {
          W(e0) = with_base ? op(SF::base(P), fp) : fp;
          W(e0 + 1) = with_base ? op(SF::base(P), fm) : fm;
        } else {
          const int n = 1 << i;
          for (int t = 0; t < n; ++t) {
            const double v = W(e0 + t);
            W(e0 + t + n) = op(v, fm);
            W(e0 + t) = op(v, fp);
          }
        }
      }
    };
    chains(Ly.A, 0, pa, SF::kBase);
    if (pb) chains(Ly.B, pa, pb, false);
    if (pc) chains(Ly.C, pa + pb, pc, false);
  } else {
    // 1. lanes over the axes: phi at the centre; the raw phi at
    //    c +- lambda3 h parked in R
    for (int k = lane; k < d; k += T) {
      double c, h;
      ch(k, c, h);
      W(Ly.phiC + k) = SF::phi(P, k, c);
      W(Ly.R + 2 * k) = SF::phi(P, k, fma(lam3, h, c));
      W(Ly.R + 2 * k + 1) = SF::phi(P, k, fma(-lam3, h, c));
    }
    group_sync<T>(mask);
    // 2. lane 0: the chains along the axes (suf, R, the centre's S, pre)
    //    and the flag masks
    if (lane == 0) {
      double suf = 0.0;
      for (int k = d - 1; k >= 0; --k) {
        const double fck = W(Ly.phiC + k);
        if (k == d - 1) {
          suf = fck;
        } else {
          W(Ly.R + 2 * k) = op(W(Ly.R + 2 * k), suf);
          W(Ly.R + 2 * k + 1) = op(W(Ly.R + 2 * k + 1), suf);
          W(Ly.suf + k) = suf;
          suf = op(fck, suf);
        }
      }
      W(Ly.sc) = SF::kBase ? op(SF::base(P), suf) : suf;
      double pre = SF::kBase ? SF::base(P) : 0.0;
      bool hp = SF::kBase;
      for (int k = 0; k < d; ++k) {
        if (hp) W(Ly.pre + k) = pre;
        const double fck = W(Ly.phiC + k);
        pre = hp ? op(pre, fck) : fck;
        hp = true;
      }
      if constexpr (SF::kFlag) {
        for (int k = 0; k < d; ++k) {
          double c, h;
          ch(k, c, h);
          zc |= (unsigned)SF::flag(P, k, c) << k;
          z3 |= ((unsigned)SF::flag(P, k, fma(lam3, h, c)) << k) |
                ((unsigned)SF::flag(P, k, fma(-lam3, h, c)) << (k + 16));
          z5 |= ((unsigned)SF::flag(P, k, fma(lam5, h, c)) << k) |
                ((unsigned)SF::flag(P, k, fma(-lam5, h, c)) << (k + 16));
        }
        W(Ly.Z) = __longlong_as_double(((long long)z3 << 32) | zc);
        W(Ly.Z + 1) = __longlong_as_double((long long)z5);
      }
    }
    group_sync<T>(mask);
    if constexpr (SF::kFlag) {
      const long long z0 = __double_as_longlong(W(Ly.Z));
      zc = (unsigned)z0;
      z3 = (unsigned)(z0 >> 32);
      z5 = (unsigned)__double_as_longlong(W(Ly.Z + 1));
    }
    // 3. lanes over the tasks: the centre and axis-node values, the
    //    pair-node prefixes L and every class-5 chain (each from its first
    //    axis, left to right: the same chains the doubling forms)
    const int na = 1 + 4 * d, nA = 1 << pa, nB = pb ? 1 << pb : 0, nC = pc ? 1 << pc : 0;
    const int ntask = na + 2 * d + nA + nB + nC;
    for (int t = lane; t < ntask; t += T) {
      if (t == 0) {
        W(Ly.fv + 4 * d) = fval(W(Ly.sc), zc != 0u);
      } else if (t < na) {
        const int k = (t - 1) >> 2, r = (t - 1) & 3;
        double c, h;
        ch(k, c, h);
        const double x = fma(lam_row(r), h, c);
        const double ph = SF::phi(P, k, x);
        const double lp = (k > 0 || SF::kBase) ? op(W(Ly.pre + k), ph) : ph;
        bool zero = false;
        if constexpr (SF::kFlag) zero = ((zc & ~(1u << k)) != 0u) || SF::flag(P, k, x);
        W(Ly.fv + r * d + k) = fval(k < d - 1 ? op(lp, W(Ly.suf + k)) : lp, zero);
      } else if (t < na + 2 * d) {
        const int e = t - na, k = e >> 1;
        double c, h;
        ch(k, c, h);
        const double ph = SF::phi(P, k, fma((e & 1) ? -lam3 : lam3, h, c));
        W(Ly.L + e) = (k > 0 || SF::kBase) ? op(W(Ly.pre + k), ph) : ph;
      } else {
        int e = t - na - 2 * d, e0 = Ly.A, j0 = 0, nb = pa;
        bool with_base = SF::kBase;
        if (e >= nA) {
          e -= nA;
          e0 = Ly.B;
          j0 = pa;
          nb = pb;
          with_base = false;
          if (e >= nB) {
            e -= nB;
            e0 = Ly.C;
            j0 = pa + pb;
            nb = pc;
          }
        }
        double acc = 0.0;
        for (int i = 0; i < nb; ++i) {
          double c, h;
          ch(j0 + i, c, h);
          const double ph = SF::phi(P, j0 + i, fma(((e >> i) & 1) ? -lam5 : lam5, h, c));
          acc = i == 0 ? (with_base ? op(SF::base(P), ph) : ph) : op(acc, ph);
        }
        W(e0 + e) = acc;
      }
    }
    group_sync<T>(mask);
    f0 = W(Ly.fv + 4 * d);
    const double two_f0 = __dmul_rn(2.0, f0);
    for (int k = lane; k < d; k += T) {
      const double t1 = __dsub_rn(__dadd_rn(W(Ly.fv + k), W(Ly.fv + d + k)), two_f0);
      const double tt = __dsub_rn(__dadd_rn(W(Ly.fv + 2 * d + k), W(Ly.fv + 3 * d + k)), two_f0);
      const double D = fabs(__dsub_rn(t1, __dmul_rn(ratio, tt)));
      if (D > dbest) {
        dbest = D;
        kbest = k;
      }
    }
    // argmax over the lanes: larger D wins, the lower axis on ties (for
    // T = 128 every axis k < d <= 16 sits in warp 0, which holds the answer
    // for lane 0, the only lane that uses it)
    constexpr int WL = T < 32 ? T : 32;
#pragma unroll
    for (int off = WL / 2; off > 0; off >>= 1) {
      const double od = __shfl_xor_sync(mask, dbest, off, WL);
      const int ok = __shfl_xor_sync(mask, kbest, off, WL);
      if (od > dbest || (od == dbest && ok < kbest)) {
        dbest = od;
        kbest = ok;
      }
    }
    // classes 2 and 3 hold 2d <= 32 nodes: one node per chunk
    PairTree t2, t3;
    const int p0 = lane_first_chunk<T>(lane), p1 = min(p0 + kChunks / T, 2 * d);
    for (int p = p0; p < p1; ++p) {
      t2.push(W(Ly.fv + (p & 1) * d + (p >> 1)));
      t3.push(W(Ly.fv + (2 + (p & 1)) * d + (p >> 1)));
    }
    bool pr2, pr3;
    const double x2 = t2.flush(pr2), x3 = t3.flush(pr3);
    s2 = lanes_tree<T>(x2, pr2, mask);
    s3 = lanes_tree<T>(x3, pr3, mask);
  }
  // class 4: c +- lambda4 h_j e_j +- lambda4 h_k e_k, j < k (lambda4 =
  // lambda3), pairs in lexicographic order, signs ++, +-, -+, --.  A lane
  // walks consecutive nodes, so mid_jk grows by one term from pair (j, k-1)
  // to (j, k) and the prefix (+) mid is shared by a pair's two nodes with
  // the same sign on j; a lane starting inside the walk forms mid_jk from
  // its first term, the same chain.
  int mj = -1, mk = -1, lp = -1, lsj = -1;
  double mid = 0.0, lm = 0.0;
  bool hmid = false;
  o.s4 = class_sum<T>(2 * d * (d - 1), lane, mask, [&](int q) -> double {
    const int p = q >> 2;
    const unsigned pr = pairs[p];
    const int j = (int)(pr >> 8), k = (int)(pr & 255u);
    const int sj = (q >> 1) & 1, sk = q & 1;
    if (p != lp) {
      if (j == mj && k == mk + 1) {
        const double t = W(Ly.phiC + mk);
        mid = hmid ? op(mid, t) : t;
        hmid = true;
      } else {
        hmid = false;
        for (int i = j + 1; i < k; ++i) {
          const double t = W(Ly.phiC + i);
          mid = hmid ? op(mid, t) : t;
          hmid = true;
        }
      }
      mj = j;
      mk = k;
      lp = p;
      lsj = -1;
    }
    if (sj != lsj) {
      const double L = W(Ly.L + 2 * j + sj);
      lm = hmid ? op(L, mid) : L;
      lsj = sj;
    }
    bool zero = false;
    if constexpr (SF::kFlag)
      zero = ((zc & ~((1u << j) | (1u << k))) != 0u) || ((z3 >> (j + 16 * sj)) & 1u) ||
             ((z3 >> (k + 16 * sk)) & 1u);
    return fval(op(lm, W(Ly.R + 2 * k + sk)), zero);
  });
  // class 5: c + lambda5 (sigma o h) for the 2^d sign patterns (bit j of m
  // set: -lambda5 on axis j); B (+) C changes every 2^a nodes
  const int am = (1 << pa) - 1, bm = (1 << pb) - 1;
  const unsigned dmask = (1u << d) - 1u;
  int mh = -1;
  double bc = 0.0;
  o.s5 = class_sum<T>(1 << d, lane, mask, [&](int m) -> double {
    double S = W(Ly.A + (m & am));
    if (pb) {
      const int hi = m >> pa;
      if (hi != mh) {
        bc = pc ? op(W(Ly.B + (hi & bm)), W(Ly.C + (hi >> pb))) : W(Ly.B + hi);
        mh = hi;
      }
      S = op(S, bc);
    }
    bool zero = false;
    if constexpr (SF::kFlag)
      zero = ((((unsigned)~m & z5) | ((unsigned)m & (z5 >> 16))) & dmask) != 0u;
    return fval(S, zero);
  });
  o.s1 = f0;
  o.s2 = s2;
  o.s3 = s3;
  o.f0 = f0;
  o.dbest = dbest;
  o.kbest = kbest;
}

// Node-wise evaluation (GMQ_EVAL_NODEWISE): the same class sums and
// fourth-difference argmax with f evaluated at every node from its
// coordinates, d operations per node for the inner chain, as an integrand
// without the separable form would be.  tab(row, j) is the region's node
// coordinate on axis j for XRow `row`; pairs[p] = (j << 8) | k for the p-th
// pair j < k of dimension d; fv points at the region's column of a
// [4d + 1] x fvs scratch array (T > 1 only).
template <int FAM, int T, class PT, class Tab>
__device__ __forceinline__ void region_sums64_nodewise(const PT& P, int d,
                                                       const unsigned short* pairs, const Tab& tab,
                                                       double* fv, int fvs, double ratio,
                                                       RegionSums& o) {
  const int lane = (T == 1) ? 0 : (int)(threadIdx.x & (unsigned)(T - 1));
  const unsigned mask = group_mask<T>();
  const int na = 1 + 4 * d;  // centre and axis nodes
  double f0 = 0.0, dbest = -1.0, s2, s3;
  int kbest = 0;
  if (T == 1) {
    PairTree t2, t3;
    double q0 = 0.0, q1 = 0.0, q2 = 0.0;
    for (int i = 0; i < na; ++i) {
      int k1 = -1, r1 = kXC, w = 0;
      if (i > 0) {
        k1 = (i - 1) >> 2;
        w = (i - 1) & 3;
        r1 = kXP2 + w;
      }
      const double v = Family<FAM>::template eval<double>(
          P, d, [&](int j) -> double { return tab(j == k1 ? r1 : kXC, j); });
      if (i == 0) {
        f0 = v;
        continue;
      }
      if (w < 2)
        t2.push(v);
      else
        t3.push(v);
      if (w == 0) {
        q0 = v;
      } else if (w == 1) {
        q1 = v;
      } else if (w == 2) {
        q2 = v;
      } else {
        const double two_f0 = __dmul_rn(2.0, f0);
        const double t1 = __dsub_rn(__dadd_rn(q0, q1), two_f0);
        const double tt = __dsub_rn(__dadd_rn(q2, v), two_f0);
        const double D = fabs(__dsub_rn(t1, __dmul_rn(ratio, tt)));
        if (D > dbest) {
          dbest = D;
          kbest = k1;
        }
      }
    }
    bool pr;
    s2 = t2.flush(pr);
    s3 = t3.flush(pr);
  } else {
    for (int i = lane; i < na; i += T) {
      int k1 = -1, r1 = kXC, w = 0;
      if (i > 0) {
        k1 = (i - 1) >> 2;
        w = (i - 1) & 3;
        r1 = kXP2 + w;
      }
      const double v = Family<FAM>::template eval<double>(
          P, d, [&](int j) -> double { return tab(j == k1 ? r1 : kXC, j); });
      fv[(i == 0 ? 4 * d : w * d + k1) * fvs] = v;
    }
    group_sync<T>(mask);
    f0 = fv[4 * d * fvs];
    const double two_f0 = __dmul_rn(2.0, f0);
    for (int k = lane; k < d; k += T) {
      const double t1 = __dsub_rn(__dadd_rn(fv[(0 * d + k) * fvs], fv[(1 * d + k) * fvs]), two_f0);
      const double tt = __dsub_rn(__dadd_rn(fv[(2 * d + k) * fvs], fv[(3 * d + k) * fvs]), two_f0);
      const double D = fabs(__dsub_rn(t1, __dmul_rn(ratio, tt)));
      if (D > dbest) {
        dbest = D;
        kbest = k;
      }
    }
    // argmax over the lanes: larger D wins, the lower axis on ties (for
    // T = 128 every axis k < d <= 16 sits in warp 0, which holds the answer
    // for lane 0, the only lane that uses it)
    constexpr int W = T < 32 ? T : 32;
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
      const double od = __shfl_xor_sync(mask, dbest, off, W);
      const int ok = __shfl_xor_sync(mask, kbest, off, W);
      if (od > dbest || (od == dbest && ok < kbest)) {
        dbest = od;
        kbest = ok;
      }
    }
    // classes 2 and 3 hold 2d <= 32 nodes: one node per chunk
    PairTree t2, t3;
    const int p0 = lane_first_chunk<T>(lane), p1 = min(p0 + kChunks / T, 2 * d);
    for (int p = p0; p < p1; ++p) {
      t2.push(fv[((p & 1) * d + (p >> 1)) * fvs]);
      t3.push(fv[((2 + (p & 1)) * d + (p >> 1)) * fvs]);
    }
    bool pr2, pr3;
    const double x2 = t2.flush(pr2), x3 = t3.flush(pr3);
    s2 = lanes_tree<T>(x2, pr2, mask);
    s3 = lanes_tree<T>(x3, pr3, mask);
  }
  // class 4: c +- lambda4 h_j e_j +- lambda4 h_k e_k, j < k
  o.s4 = class_sum<T>(2 * d * (d - 1), lane, mask, [&](int q) -> double {
    const unsigned pr = pairs[q >> 2];
    const int kj = (int)(pr >> 8), kk = (int)(pr & 255u);
    const int rj = (q & 2) ? kXM3 : kXP3, rk = (q & 1) ? kXM3 : kXP3;
    return Family<FAM>::template eval<double>(
        P, d, [&](int j) -> double { return tab(j == kj ? rj : (j == kk ? rk : kXC), j); });
  });
  // class 5: c + lambda5 (sigma o h) for the 2^d sign patterns
  o.s5 = class_sum<T>(1 << d, lane, mask, [&](int m) -> double {
    return Family<FAM>::template eval<double>(P, d, [&](int j) -> double {
      return tab((((unsigned)m >> j) & 1u) ? kXM5 : kXP5, j);
    });
  });
  o.s1 = f0;
  o.s2 = s2;
  o.s3 = s3;
  o.f0 = f0;
  o.dbest = dbest;
  o.kbest = kbest;
}

// Null-rule error estimate of a region from its class sums (the heuristic
// of Berntsen, Espelid & Genz 1991 that the paper's Sec. 2 cites; constants
// and combination as the library reads it).  nw: 4 x 5 per-node weights of
// four fully symmetric null rules on the rule's node classes (degrees 5,
// 3, 3, 1, mutually orthogonal, each with the norm of the degree-7
// weights; unit volume).  N_k = vol sum_c nw[k][c] S_c; e1 = |N1|,
// e2 = sqrt(N2^2 + N3^2), e3 = |N4|; r = max(e1 / e2, e2 / e3) (x / 0 = inf
// for x > 0, 0 / 0 = 0) is the decay per degree step.  r >= 1 (not yet
// asymptotic): 10 max(e); r < 1: 10 r e1, e1 extrapolated by one decay step
// (the degree-5 null rule is one step below the degree-7 rule).  Every
// operation is rounded separately, in the order written.
__device__ __forceinline__ double null_ratio(double x, double y) {
  if (y > 0.0) return __ddiv_rn(x, y);
  return x > 0.0 ? __longlong_as_double(0x7ff0000000000000ll) : 0.0;
}

__device__ __forceinline__ double null_rule_estimate(const RegionSums& o, double vol,
                                                     const double* nw) {
  const double s[5] = {o.s1, o.s2, o.s3, o.s4, o.s5};
  double nul[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double t = __dmul_rn(nw[k * 5], s[0]);
#pragma unroll
    for (int c = 1; c < 5; ++c) t = __dadd_rn(t, __dmul_rn(nw[k * 5 + c], s[c]));
    nul[k] = __dmul_rn(vol, t);
  }
  const double e1 = fabs(nul[0]);
  const double e2 = __dsqrt_rn(__dadd_rn(__dmul_rn(nul[1], nul[1]), __dmul_rn(nul[2], nul[2])));
  const double e3 = fabs(nul[3]);
  const double r = fmax(null_ratio(e1, e2), null_ratio(e2, e3));
  if (r >= 1.0) return __dmul_rn(10.0, fmax(e1, fmax(e2, e3)));
  return __dmul_rn(__dmul_rn(10.0, r), e1);
}

// 2 h, exactly: for normal h one more in the exponent field (integer work,
// which keeps the FP64 pipe free), the multiplication otherwise (zero,
// subnormal, or 2 h overflowing).
__device__ __forceinline__ double twice_exact(double h) {
  const int hi = __double2hiint(h);
  const unsigned ex = ((unsigned)hi >> 20) & 0x7ffu;
  if (ex - 1u < 2045u) return __hiloint2double(hi + (1 << 20), __double2loint(h));
  return __dmul_rn(2.0, h);
}

// Rule values, error estimate, split axis and round-off guard of a region
// from its class sums (one lane).  cval(k), hval(k): centre and half-width.
// nw: the null-rule table for the null-rule estimate, or null for the
// embedded estimate |I7 - I5|.
template <class CV, class HV>
__device__ __forceinline__ void region_finish64(const RegionSums& o, int d, const double* w7,
                                                const double* w5, const double* nw,
                                                double vol_omega, CV cval, HV hval, double* i7o,
                                                double* erro, double* vfo, uint8_t* axo) {
  double vol = 1.0;
  for (int k = 0; k < d; ++k) vol = __dmul_rn(vol, twice_exact(hval(k)));
  double t7 = __dmul_rn(w7[0], o.s1);
  t7 = __dadd_rn(t7, __dmul_rn(w7[1], o.s2));
  t7 = __dadd_rn(t7, __dmul_rn(w7[2], o.s3));
  t7 = __dadd_rn(t7, __dmul_rn(w7[3], o.s4));
  t7 = __dadd_rn(t7, __dmul_rn(w7[4], o.s5));
  double t5 = __dmul_rn(w5[0], o.s1);
  t5 = __dadd_rn(t5, __dmul_rn(w5[1], o.s2));
  t5 = __dadd_rn(t5, __dmul_rn(w5[2], o.s3));
  t5 = __dadd_rn(t5, __dmul_rn(w5[3], o.s4));
  const double i7 = __dmul_rn(vol, t7);
  const double i5 = __dmul_rn(vol, t5);
  // split axis: flat differences -> the widest axis (lowest index on ties)
  const double flat_thr = __dadd_rn(__dmul_rn(1e-14, fabs(o.f0)), 1e-300);
  int ax = o.kbest;
  if (!(o.dbest > flat_thr)) {
    ax = 0;
    double hb = hval(0);
    for (int k = 1; k < d; ++k) {
      const double hk = hval(k);
      if (hk > hb) {
        hb = hk;
        ax = k;
      }
    }
  }
  // round-off guard: bisection along ax must move the centre
  const double cs = cval(ax);
  const double hh = __dmul_rn(0.5, hval(ax));
  const bool bad = (hh == 0.0) || (__dsub_rn(cs, hh) == cs) || (__dadd_rn(cs, hh) == cs);
  *i7o = i7;
  *erro = nw ? null_rule_estimate(o, vol, nw) : fabs(__dsub_rn(i7, i5));
  if (vfo) {
    // vol / vol(Omega); a unit domain (bits of 1.0) divides by one
    const bool unit = __double_as_longlong(vol_omega) == 0x3ff0000000000000ll;
    *vfo = unit ? vol : __ddiv_rn(vol, vol_omega);
  }
  *axo = (uint8_t)(ax | (bad ? 0x80 : 0));
}

}  // namespace gmq
