"""Fully symmetric null rules on the Genz-Malik node set, for the oracle's
Berntsen-Espelid-Genz error estimate, computed in exact rational arithmetic.

Test infrastructure only (see gm_oracle.h): the CUDA library computes its own
copy of these weights independently, in floating point on the host.

The paper (Sec. 2, error estimator) names the heuristic of Berntsen, Espelid
and Genz (ACM TOMS 17, 1991) without printing it.  Its ingredients, as this
project reads them:

* A null rule is a weighted sum over the basic rule's own nodes whose value
  is zero for every polynomial up to some degree (its weights sum to zero).
  It costs nothing extra: it reuses the integrand values of the rule.
* Fully symmetric null rules give one weight per node class (centre,
  +-lambda2 e_k, +-lambda3 e_k, +-lambda4 e_j +-lambda4 e_k, the 2^d
  (+-lambda5, ...) corners), so their values are linear combinations of the
  five class sums S_1..S_5 that the rule already forms.
* By symmetry every odd monomial vanishes on every such rule; the even
  conditions up to degree 5 are the orbit sums of 1, x_1^2, x_1^4 and
  x_1^2 x_2^2.  With lambda^2 rational (9/70, 9/10, 9/10, 9/19) all of them
  are exact rationals.  On five classes the null rules of degree >= 5 form a
  space of dimension 1, those of degree >= 3 one of dimension 3 and those of
  degree >= 1 one of dimension 4 (d >= 2; for d = 1, with no pair class,
  1, 2 and 3).
* The null rules are made mutually orthogonal for the inner product of
  their node weights, <u, v> = sum over nodes u(x) v(x) = sum_c n_c u_c v_c
  (n_c = nodes in class c), in order of decreasing degree (Gram-Schmidt:
  N1 spans the degree-5 space, N2, N3 complete the degree-3 space, N4 the
  degree-1 space), and each is scaled to the norm of the basic rule's
  weights, <N, N> = <w7, w7>.

The table for dimension d is 4 x 5 doubles: row k holds N_{k+1}'s weight
per node of classes 1..5, normalised to a unit-volume region as the rule's
weights are (value = vol * sum_c N_c S_c).  For d = 1, N3 does not exist
(its row is zero) and the pair class has no node (weight 0).
"""
from __future__ import annotations

from fractions import Fraction as F
from functools import lru_cache
from math import isqrt

LAM2 = {2: F(9, 70), 3: F(9, 10), 4: F(9, 10), 5: F(9, 19)}  # lambda_g^2


def class_sizes(d: int) -> list[int]:
    """Nodes per class: centre, +-lambda2 e_k, +-lambda3 e_k, pairs, corners."""
    return [1, 2 * d, 2 * d, 2 * d * (d - 1), 2 ** d]


def basic_weights(d: int) -> list[F]:
    """The degree-7 rule's weight per node of each class, unit volume
    (Genz & Malik 1980)."""
    return [F(12824 - 9120 * d + 400 * d * d, 19683), F(980, 6561), F(1820 - 400 * d, 19683),
            F(200, 19683), F(6859, 19683 * 2 ** d)]


def moment_rows(d: int) -> dict[str, list[F]]:
    """Class sums of the even monomials up to degree 4 (rows of the
    conditions; entry c is the sum of the monomial over class c's nodes)."""
    l2, l3, l4, l5 = LAM2[2], LAM2[3], LAM2[4], LAM2[5]
    rows = {"1": [F(n) for n in class_sizes(d)],
            "x1^2": [F(0), 2 * l2, 2 * l3, 4 * (d - 1) * l4, 2 ** d * l5],
            "x1^4": [F(0), 2 * l2 ** 2, 2 * l3 ** 2, 4 * (d - 1) * l4 ** 2, 2 ** d * l5 ** 2]}
    if d >= 2:
        rows["x1^2x2^2"] = [F(0), F(0), F(0), 4 * l4 ** 2, 2 ** d * l5 ** 2]
    return rows


def _null_space(rows: list[list[F]], cols: list[int]) -> list[list[F]]:
    """Basis of {v : row . v = 0 for every row, v_c = 0 outside cols}, by
    exact reduced row echelon form over the columns in cols."""
    m = [[r[c] for c in cols] for r in rows]
    piv = []
    ri = 0
    for ci in range(len(cols)):
        p = next((i for i in range(ri, len(m)) if m[i][ci] != 0), None)
        if p is None:
            continue
        m[ri], m[p] = m[p], m[ri]
        inv = 1 / m[ri][ci]
        m[ri] = [x * inv for x in m[ri]]
        for i in range(len(m)):
            if i != ri and m[i][ci] != 0:
                f = m[i][ci]
                m[i] = [x - f * y for x, y in zip(m[i], m[ri])]
        piv.append(ci)
        ri += 1
    free = [ci for ci in range(len(cols)) if ci not in piv]
    basis = []
    for fc in free:
        v = [F(0)] * len(cols)
        v[fc] = F(1)
        for i, pc in enumerate(piv):
            v[pc] = -m[i][fc]
        full = [F(0)] * 5
        for k, c in enumerate(cols):
            full[c] = v[k]
        basis.append(full)
    return basis


def inner(d: int, u: list[F], v: list[F]) -> F:
    return sum((n * a * b for n, a, b in zip(class_sizes(d), u, v)), F(0))


@lru_cache(maxsize=None)
def null_rules_exact(d: int) -> tuple:
    """(orthogonal null rules N1..N4 before scaling, their degrees): exact
    rationals, N3 absent (None) for d = 1."""
    rows = moment_rows(d)
    cols = [0, 1, 2, 3, 4] if d >= 2 else [0, 1, 2, 4]
    deg5 = _null_space([rows[k] for k in rows], cols)
    deg3 = _null_space([rows["1"], rows["x1^2"]], cols)
    deg1 = _null_space([rows["1"]], cols)
    out = []

    def add(cands):
        for v in cands:
            w = list(v)
            for q in out:
                f = inner(d, w, q) / inner(d, q, q)
                w = [a - f * b for a, b in zip(w, q)]
            if any(x != 0 for x in w):
                out.append(w)
                return True
        return False

    assert add(deg5) and len(deg5) == 1
    degrees = [5]
    for _ in range(2 if d >= 2 else 1):
        assert add(deg3)
        degrees.append(3)
    assert add(deg1)
    degrees.append(1)
    if d == 1:
        out.insert(2, None)
        degrees.insert(2, None)
    return tuple(tuple(v) if v is not None else None for v in out), tuple(degrees)


def _sqrt_ratio(p: F, bits: int = 200) -> F:
    """sqrt(p) for a positive rational p, to 2^-bits relative (integer
    square root of the scaled numerator and denominator)."""
    num = isqrt(p.numerator * (1 << (2 * bits)) * p.denominator)
    return F(num, p.denominator * (1 << bits))


def null_table(d: int) -> list[float]:
    """The 4 x 5 weight table (row-major) of the scaled null rules for
    dimension d, each weight rounded once to the nearest double."""
    rules, _ = null_rules_exact(d)
    w7 = basic_weights(d)
    target = inner(d, w7, w7)
    out = []
    for v in rules:
        if v is None:
            out.extend([0.0] * 5)
            continue
        s = _sqrt_ratio(target / inner(d, v, v))
        out.extend(float(x * s) for x in v)
    return out
