"""Pins of the oracle's null-rule error estimate (paper Sec. 2 cites the
Berntsen-Espelid-Genz heuristic; oracle/null_rules.py builds the null rules,
or_null_estimate in oracle/gm_oracle.c combines them).

Each pin checks something other than the construction itself: the null
rules against every monomial on the explicit node set (not the orbit
sums), the one-dimensional degree-5 null rule against the divided-difference
weights, the degree-5 rule against the embedded-rule difference, the
combination against hand-worked values, the rounding band against
perturbed class sums, and the estimate against true errors of boxes with
closed-form integrals.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G

LAM = [math.sqrt(9 / 70), math.sqrt(9 / 10), math.sqrt(9 / 10), math.sqrt(9 / 19)]


def _nodes(d):
    """Explicit Genz-Malik nodes on [-1, 1]^d with their class index (0..4),
    written out from the generator definitions."""
    out = [(np.zeros(d), 0)]
    for cls, lam in ((1, LAM[0]), (2, LAM[1])):
        for k in range(d):
            for s in (1, -1):
                x = np.zeros(d)
                x[k] = s * lam
                out.append((x, cls))
    for j, k in itertools.combinations(range(d), 2):
        for sj, sk in itertools.product((1, -1), repeat=2):
            x = np.zeros(d)
            x[j], x[k] = sj * LAM[2], sk * LAM[2]
            out.append((x, 3))
    for signs in itertools.product((1, -1), repeat=d):
        out.append((LAM[3] * np.array(signs, dtype=float), 4))
    return out


def _monomials(d, deg):
    return [a for a in itertools.product(range(deg + 1), repeat=d) if sum(a) == deg]


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_null_rules_annihilate_exactly_their_degree(oracle, d):
    W = oracle.null_table(d).reshape(4, 5)
    nodes = _nodes(d)
    assert len(nodes) == oracle.num_nodes(d)
    X = np.array([x for x, _ in nodes])
    cls = np.array([c for _, c in nodes])
    for k, deg in enumerate((5, 3, 3, 1)):
        if d == 1 and k == 2:
            assert np.all(W[k] == 0.0)  # one dimension: no second degree-3 rule
            continue
        w = W[k][cls]
        assert abs(w.sum()) <= 1e-14
        for p in range(1, deg + 1):
            for a in _monomials(d, p):
                v = np.prod(X ** np.array(a), axis=1) @ w
                assert abs(v) <= 1e-14, (k, a, v)
        # and not the next degree: some monomial of degree deg + 1 survives
        top = max(abs(np.prod(X ** np.array(a), axis=1) @ w) for a in _monomials(d, deg + 1))
        assert top > 1e-3, (k, top)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_null_rules_orthogonal_with_the_basic_rules_norm(oracle, d):
    W = oracle.null_table(d).reshape(4, 5)
    w7, _ = oracle.weights(d)
    nodes = _nodes(d) if d <= 5 else None
    n = np.array([1, 2 * d, 2 * d, 2 * d * (d - 1), 2 ** d], dtype=float)
    if nodes is not None:
        counts = np.bincount([c for _, c in nodes], minlength=5)
        assert np.array_equal(counts, n)
    norm7 = np.sum(n * w7 * w7)
    rows = [0, 1, 3] if d == 1 else [0, 1, 2, 3]
    for i in rows:
        assert abs(np.sum(n * W[i] * W[i]) - norm7) <= 1e-14 * norm7
        for j in rows:
            if j != i:
                assert abs(np.sum(n * W[i] * W[j])) <= 1e-14 * norm7


def test_d1_degree5_null_rule_is_the_divided_difference(oracle):
    """On seven distinct points the only functional that vanishes on every
    polynomial of degree <= 5 is the sixth divided difference, weights
    1 / prod_{j != i} (x_i - x_j)."""
    W = oracle.null_table(1).reshape(4, 5)
    nodes = _nodes(1)
    x = np.array([p[0][0] for p in nodes])
    dd = np.array([1.0 / np.prod([xi - xj for xj in x if xj != xi]) for xi in x])
    w = W[0][[c for _, c in nodes]]
    ratio = w / dd
    assert np.allclose(ratio, ratio[0], rtol=1e-12, atol=0)


@pytest.mark.parametrize("fam", [G.GAUSSIAN, G.OSCILLATORY, G.C0, G.PRODUCT_PEAK])
def test_degree5_null_rule_is_the_embedded_difference(oracle, fam):
    """I7 - I5 vanishes to degree 5 too, so it is the degree-5 null rule up to
    its norm: e1 = |w7| / |w7 - w5| * |I7 - I5| on every region."""
    d = 4
    a, u = G.seed_genz(2, fam, d, G.GENZ_TARGET_SUM.get(fam, 12.0))
    w7, w5 = oracle.weights(d)
    n = np.array([1, 2 * d, 2 * d, 2 * d * (d - 1), 2 ** d], dtype=float)
    f = math.sqrt(np.sum(n * w7 * w7) / np.sum(n * (w7 - w5) ** 2))
    c, h = G.random_boxes(31, 40, d)
    for k in range(len(c)):
        r = oracle.rule(c[k], h[k], family=fam, a=a, u=u)
        q = oracle.null_estimate(r, d)
        mag = r.vol * np.sum(r.sabs)
        assert abs(q["e"][0] - f * abs(r.i7 - r.i5)) <= 1e-12 * mag


def _rule_with_nulls(oracle, d, nul, vol=1.0):
    """A rule result whose class sums give the four null values `nul`
    (least-norm class sums; the w7 direction is left at zero)."""
    W = oracle.null_table(d).reshape(4, 5)
    s = np.linalg.pinv(W) @ (np.asarray(nul, dtype=float) / vol)
    r = oracle.rule(np.full(d, 0.5), np.full(d, 0.5), f=lambda x: 0.0)
    raw = r._raw
    for c in range(5):
        raw.s[c] = s[c]
        raw.sabs[c] = abs(s[c])
    raw.vol = vol
    return r


@pytest.mark.parametrize("nul,regime,want", [
    # e = (1e-3, 1e-2, 1e-1): r = 0.1, asymptotic: 10 * 0.1 * 1e-3
    ((1e-3, 0.006, 0.008, 0.1), 1, 1e-3),
    # e = (0.1, 0.15, 0.2): r = 0.75: 10 * 0.75 * 0.1
    ((0.1, 0.09, 0.12, 0.2), 1, 0.75),
    # e = (0.3, 0.2, 0.5): r = 1.5, not asymptotic: 10 * max(e)
    ((0.3, 0.12, -0.16, 0.5), 0, 5.0),
    # all zero: the rule is exact on f's node values
    ((0.0, 0.0, 0.0, 0.0), 1, 0.0),
    # only the degree-1 rule sees f (f linear plus degree-2 content): r = 0
    ((0.0, 0.0, 0.0, 0.7), 1, 0.0),
    # e2 = 0 < e1: r = infinity
    ((0.25, 0.0, 0.0, 0.0), 0, 2.5),
])
def test_combination_hand_cases(oracle, nul, regime, want):
    d = 3
    q = oracle.null_estimate(_rule_with_nulls(oracle, d, nul), d)
    assert np.allclose(q["nul"], nul, rtol=1e-12, atol=1e-15)
    assert q["regime"] == regime
    assert abs(q["est"] - want) <= 1e-12 * max(want, 1.0)


def test_regime_boundary_is_flagged(oracle):
    d = 3
    # r = 1 exactly (e1 = e2): the estimate jumps from 10 e1 to 10 max(e)
    q = oracle.null_estimate(_rule_with_nulls(oracle, d, (0.2, 0.12, 0.16, 0.9)), d)
    assert q["r"] == pytest.approx(1.0, rel=1e-12) and q["regime_tie"]
    assert {round(q["est"], 9), round(q["est_alt"], 9)} == {2.0, 9.0}
    # far from the boundary: no flag
    q = oracle.null_estimate(_rule_with_nulls(oracle, d, (0.02, 0.12, 0.16, 0.9)), d)
    assert not q["regime_tie"]


@pytest.mark.parametrize("fam,d", [(G.GAUSSIAN, 3), (G.OSCILLATORY, 5), (G.CORNER_PEAK, 8),
                                   (G.C0, 4), (G.PRODUCT_PEAK, 2)])
def test_band_covers_other_summation_orders(oracle, fam, d):
    """Class sums added in another order differ by at most about n 2^-53 of
    their magnitude; perturbing them by that much (n = the class size, each
    sign at random) moves the estimate by less than its band, or to its
    other regime's value when the band reaches across r = 1."""
    a, u = G.seed_genz(3, fam, d, G.GENZ_TARGET_SUM.get(fam, 5.0 * d))
    c, h = G.random_boxes(5 + d, 60, d)
    n = np.array([1, 2 * d, 2 * d, 2 * d * (d - 1), 2 ** d], dtype=float)
    rng = np.random.default_rng(d)
    for k in range(len(c)):
        for scale in (1.0, 0.02):  # the random box and a small box at its centre
            r = oracle.rule(c[k], h[k] * scale, family=fam, a=a, u=u)
            q0 = oracle.null_estimate(r, d)
            raw = r._raw
            for _ in range(4):
                for cc in range(5):
                    raw.s[cc] = r.s[cc] + rng.choice((-1, 1)) * n[cc] * 2.0 ** -53 * r.sabs[cc]
                q = oracle.null_estimate(r, d)
                near = min(abs(q["est"] - q0["est"]),
                           abs(q["est"] - q0["est_alt"]) if q0["regime_tie"] else math.inf)
                assert near <= q0["band"], (k, scale, q["est"], q0)


def _gauss_box(mp, a, u, c, h):
    """Closed-form Gaussian integral over one box, at 40 digits (the erf
    differences of narrow boxes cancel in FP64)."""
    out = mp.mpf(1)
    for ak, uk, ck, hk in zip(a, u, c, h):
        ak, uk, ck, hk = (mp.mpf(float(v)) for v in (ak, uk, ck, hk))
        out *= mp.sqrt(mp.pi) / (2 * ak) * (mp.erf(ak * (ck + hk - uk)) - mp.erf(ak * (ck - hk - uk)))
    return out


def test_estimate_bounds_the_true_error_on_resolved_boxes(oracle):
    """On boxes where f is resolved (asymptotic regime, r < 1) the estimate
    bounds the degree-7 rule's true error (Gaussian family, closed form per
    box) on at least 95 % of the boxes and comes within 10 % of it on all,
    while it is far less pessimistic than the embedded estimate |I7 - I5|;
    and it shrinks with the box faster than the embedded estimate.  True
    errors at FP64 rounding level of the rule value itself are not compared
    (no estimate can see them)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    d = 3
    a, u = G.seed_genz(1, G.GAUSSIAN, d, 3.5)
    c, h = G.random_boxes(77, 80, d)
    ratio, ratio_emb = [], []
    for k in range(len(c)):
        for scale in (0.25, 0.1, 0.04):
            hk = h[k] * scale
            r = oracle.rule(c[k], hk, family=G.GAUSSIAN, a=a, u=u)
            q = oracle.null_estimate(r, d)
            exact = _gauss_box(mp, a, u, c[k], hk)
            true = float(abs(mp.mpf(r.i7) - exact))
            if q["regime"] == 1 and true > 1e-14 * float(abs(exact)):
                ratio.append(q["est"] / true)
                ratio_emb.append(r.err / true)
        r1 = oracle.rule(c[k], h[k] * 0.1, family=G.GAUSSIAN, a=a, u=u)
        r2 = oracle.rule(c[k], h[k] * 0.05, family=G.GAUSSIAN, a=a, u=u)
        q1, q2 = oracle.null_estimate(r1, d), oracle.null_estimate(r2, d)
        if q1["regime"] == 1 and q2["regime"] == 1 and r2.err > 1e-12 * r2.vol:
            # halving every side: null estimate ~ h^8 vol, embedded ~ h^6 vol
            assert q2["est"] / q1["est"] < 0.5 * r2.err / r1.err
    ratio, ratio_emb = np.array(ratio), np.array(ratio_emb)
    assert len(ratio) >= 80
    assert np.mean(ratio >= 1.0) >= 0.95 and ratio.min() >= 0.9
    assert np.all(ratio_emb >= 1.0)
    assert np.median(ratio) * 10 < np.median(ratio_emb)


@pytest.mark.parametrize("fam,d,tol", [(G.GAUSSIAN, 4, 1e-8), (G.OSCILLATORY, 5, 1e-7),
                                       (G.CORNER_PEAK, 4, 1e-8), (G.PRODUCT_PEAK, 3, 1e-7),
                                       (G.C0, 3, 1e-5)])
def test_loop_with_null_rules_meets_the_tolerance(oracle, fam, d, tol):
    from tests import closed_forms as CF
    a, u = G.seed_genz(4, fam, d, {G.PRODUCT_PEAK: 5.0 * d}.get(fam, G.GENZ_TARGET_SUM.get(fam)))
    ex = CF.exact(fam, a, u)
    r = oracle.integrate(fam, a, u, tol, max_regions=1 << 20, estimator=oracle.EST_NULL_RULES)
    e = oracle.integrate(fam, a, u, tol, max_regions=1 << 20)
    assert r.status == 0 and r.error <= tol * abs(r.integral)
    assert abs(r.integral - ex) <= tol * abs(ex), (r.integral, ex)
    assert r.regions_evaluated <= e.regions_evaluated * 1.5
    assert len(r.trace) == r.iterations


def test_null_rules_reject_the_gauss_kronrod_rule(oracle):
    a, u = G.seed_genz(1, G.GAUSSIAN, 2, 3.5)
    r = oracle.integrate(G.GAUSSIAN, a, u, 1e-6, rule=oracle.RULE_GK,
                         estimator=oracle.EST_NULL_RULES)
    assert r.status == -1
