"""Gauss-Kronrod (7, 15) nodes and weights on [-1, 1] for the oracle's
tensor-product rule, computed in exact rational arithmetic.

Test infrastructure only (see gm_oracle.h): the CUDA library computes its
own copy of these constants independently, by floating-point Newton
iteration on the host.

The rule (Kronrod 1965; the paper's Sec. 3 names a tensor-product
Gauss-Kronrod rule without printing it): the 7-point Gauss-Legendre rule G7
and its Kronrod extension K15, which adds the 8 zeros of the Stieltjes
polynomial E8 and has polynomial degree 3n + 1 = 22.

* Gauss nodes: the zeros of the Legendre polynomial P7 (rational
  coefficients), isolated in the intervals between the Chebyshev-like
  starting points and refined by bisection on exact values to 2^-80.
* E8 = sum_{m=0..4} a_m P_{2m} with a_4 = 1 (E8 is even because 8 is), and
  int_{-1}^{1} E8(x) P7(x) x^k dx = 0 for k = 0..7; the conditions with k
  even vanish by parity, the four with k odd fix a_0..a_3.  All integrals
  are exact (int x^p = 2 / (p + 1) for even p).
* E8's zeros interlace the Gauss nodes: one in (0, g1), (g1, g2), (g2, g3)
  and (g3, 1) for the positive Gauss nodes g1 < g2 < g3; each is found by
  bisection on exact values.
* Weights: K15's from the exactness conditions sum_i w_i P_m(x_i) = 2 d_m0,
  m = 0, 2, ..., 14 (odd m hold by symmetry), solved exactly on the
  rational node approximations; G7's from w = 2 / ((1 - x^2) P7'(x)^2).
"""
from __future__ import annotations

from fractions import Fraction as F
from functools import lru_cache


def _legendre(n: int) -> list[F]:
    """Coefficients (lowest degree first) of P_n by the three-term recurrence
    (k + 1) P_{k+1} = (2k + 1) x P_k - k P_{k-1}."""
    p0, p1 = [F(1)], [F(0), F(1)]
    if n == 0:
        return p0
    for k in range(1, n):
        nxt = [F(0)] * (k + 2)
        for i, c in enumerate(p1):
            nxt[i + 1] += F(2 * k + 1, k + 1) * c
        for i, c in enumerate(p0):
            nxt[i] -= F(k, k + 1) * c
        p0, p1 = p1, nxt
    return p1


def _mul(a: list[F], b: list[F]) -> list[F]:
    out = [F(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _integral(p: list[F]) -> F:
    """int_{-1}^{1} p(x) dx, exactly."""
    return sum((2 * c / (i + 1) for i, c in enumerate(p) if i % 2 == 0), F(0))


def _eval(p: list[F], x: F) -> F:
    v = F(0)
    for c in reversed(p):
        v = v * x + c
    return v


def _bisect(p: list[F], lo: F, hi: F, bits: int = 80) -> F:
    flo = _eval(p, lo)
    assert flo != 0 and (flo > 0) != (_eval(p, hi) > 0), "no sign change"
    for _ in range(bits):
        mid = (lo + hi) / 2
        fm = _eval(p, mid)
        if fm == 0:
            return mid
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return (lo + hi) / 2


def _solve(a: list[list[F]], b: list[F]) -> list[F]:
    """Exact Gaussian elimination."""
    n = len(b)
    m = [row[:] + [b[i]] for i, row in enumerate(a)]
    for c in range(n):
        piv = next(r for r in range(c, n) if m[r][c] != 0)
        m[c], m[piv] = m[piv], m[c]
        for r in range(n):
            if r != c and m[r][c] != 0:
                f = m[r][c] / m[c][c]
                m[r] = [x - f * y for x, y in zip(m[r], m[c])]
    return [m[i][n] / m[i][i] for i in range(n)]


def _deriv(p: list[F]) -> list[F]:
    return [i * c for i, c in enumerate(p)][1:]


@lru_cache(maxsize=None)
def gk15() -> dict:
    """Nodes (ascending, 15) and the K15 and G7 weights on [-1, 1] (G7's are
    0 at the 8 Kronrod-only nodes), as Fractions, plus `gauss_index` (the
    positions of the Gauss nodes in the node list)."""
    p7 = _legendre(7)
    # positive zeros of P7: one in each interval between the sign changes of
    # P7 on a fine grid of (0, 1)
    grid = [F(i, 64) for i in range(1, 64)] + [F(1)]
    gpos, prev = [], F(1, 64)
    for x in grid[1:]:
        if (_eval(p7, prev) > 0) != (_eval(p7, x) > 0):
            gpos.append(_bisect(p7, prev, x))
        prev = x
    assert len(gpos) == 3
    # Stieltjes polynomial E8 = sum a_m P_{2m}, a_4 = 1
    P = [_legendre(2 * m) for m in range(5)]
    rows, rhs = [], []
    for k in (1, 3, 5, 7):
        xk = [F(0)] * k + [F(1)]
        base = _mul(p7, xk)
        rows.append([_integral(_mul(P[m], base)) for m in range(4)])
        rhs.append(-_integral(_mul(P[4], base)))
    a = _solve(rows, rhs) + [F(1)]
    e8 = [F(0)] * 9
    for m in range(5):
        for i, c in enumerate(P[m]):
            e8[i] += a[m] * c
    bounds = [F(0)] + gpos + [F(1)]
    kpos = [_bisect(e8, bounds[i], bounds[i + 1]) for i in range(4)]
    pos = sorted(gpos + kpos)  # 7 positive nodes, alternating K, G, K, ...
    nodes = [-x for x in reversed(pos)] + [F(0)] + pos
    # K15 weights: w(0) and w(x) = w(-x) for the 7 positive nodes
    distinct = [F(0)] + pos
    rows, rhs = [], []
    for m in range(0, 15, 2):
        pm = _legendre(m)
        rows.append([_eval(pm, x) * (1 if x == 0 else 2) for x in distinct])
        rhs.append(F(2) if m == 0 else F(0))
    wd = _solve(rows, rhs)
    wk = [wd[1 + pos.index(-x)] for x in nodes[:7]] + [wd[0]] + [wd[1 + i] for i in range(7)]
    dp7 = _deriv(p7)
    gset = set(gpos) | {-x for x in gpos} | {F(0)}
    wg = [2 / ((1 - x * x) * _eval(dp7, x) ** 2) if x in gset else F(0) for x in nodes]
    gidx = [i for i, x in enumerate(nodes) if x in gset]
    return {"nodes": nodes, "wk": wk, "wg": wg, "gauss_index": gidx, "e8": e8, "p7": p7}


def gk15_float():
    """The same tables rounded to float (lists of 15)."""
    t = gk15()
    return ([float(x) for x in t["nodes"]], [float(x) for x in t["wk"]],
            [float(x) for x in t["wg"]])
