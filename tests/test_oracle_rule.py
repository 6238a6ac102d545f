"""Pins of the oracle's Genz-Malik rule against mathematics fixed independently
of it (paper Sec. 2: fully symmetric degree-7 rule with embedded degree-5
rule, fourth-difference axis choice).

* exactness: I7 integrates every monomial of total degree <= 7 over a box,
  I5 every monomial of degree <= 5; I7 is not exact at degree 8 and I5 is
  not exact at degree 6 (so both degrees are pinned from both sides);
* d = 1: the rule is the 7-point symmetric rule whose weights are fixed by
  the moment equations for 1, x^2, x^4, x^6 (solved here with numpy);
* node count 2^d + 2d^2 + 2d + 1 by counting the integrand calls;
* symmetry invariants (axis permutation, reflection about the centre);
* fourth differences vanish for cubics and single out the axis of x_k^4.
"""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest


def _monomials(d, deg):
    out = []
    for total in range(deg + 1):
        for combo in itertools.combinations_with_replacement(range(d), total):
            e = [0] * d
            for k in combo:
                e[k] += 1
            out.append(tuple(e))
    return out


def _exact_monomial(c, h, e):
    val = Fraction(1)
    for ck, hk, p in zip(c, h, e):
        lo = Fraction(ck) - Fraction(hk)
        hi = Fraction(ck) + Fraction(hk)
        val *= (hi ** (p + 1) - lo ** (p + 1)) / (p + 1)
    return float(val)


def _mono_fn(e):
    e = np.array(e)

    def f(x):
        return float(np.prod(x ** e))
    return f


def _box(rng, d):
    c = np.array([rng.uniform(0.2, 0.8) for _ in range(d)])
    h = np.array([rng.uniform(0.05, 0.2) for _ in range(d)])
    return c, h


def test_node_count_by_calls(oracle):
    for d in range(1, 11):
        calls = [0]

        def f(x):
            calls[0] += 1
            return 1.0
        oracle.rule(np.full(d, 0.5), np.full(d, 0.5), f=f)
        assert calls[0] == 2 ** d + 2 * d * d + 2 * d + 1 == oracle.num_nodes(d)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6])
def test_exact_all_monomials_low_d(oracle, d):
    rng = random.Random(100 + d)
    c, h = _box(rng, d)
    for e in _monomials(d, 8):
        r = oracle.rule(c, h, f=_mono_fn(e))
        ex = _exact_monomial(c, h, e)
        scale = r.vol * float(np.prod((c + h) ** np.array(e)))
        deg = sum(e)
        if deg <= 7:
            assert abs(r.i7 - ex) <= 1e-13 * scale, (e, r.i7, ex)
        if deg <= 5:
            assert abs(r.i5 - ex) <= 1e-13 * scale, (e, r.i5, ex)
    # degree 8 is beyond I7 and degree 6 beyond I5: centred powers
    # (x_1 - c_1)^p integrate to vol * h_1^p / (p + 1); the rule misses them
    # by a fixed fraction of that value
    for p, which in ((8, "i7"), (6, "i5")):
        r = oracle.rule(c, h, f=lambda x, p=p: float((x[0] - c[0]) ** p))
        ex = r.vol * h[0] ** p / (p + 1)
        assert abs(getattr(r, which) - ex) > 1e-3 * ex, (p, which)
    r = oracle.rule(c, h, f=lambda x: float((x[0] - c[0]) ** 6))
    assert abs(r.i7 - r.vol * h[0] ** 6 / 7) <= 1e-13 * r.vol * h[0] ** 6


@pytest.mark.parametrize("d", [7, 8, 10, 12])
def test_exact_sampled_monomials_high_d(oracle, d):
    rng = random.Random(200 + d)
    c, h = _box(rng, d)
    monos = _monomials(d, 7)
    rng.shuffle(monos)
    # every pair-class and sign-class node must matter: keep monomials that
    # mix several axes with even and odd powers
    picked = monos[: (60 if d <= 8 else 12)]
    picked.append(tuple([1] * 7 + [0] * (d - 7)))
    picked.append(tuple([2, 2, 2] + [0] * (d - 3)))
    for e in picked:
        r = oracle.rule(c, h, f=_mono_fn(e))
        ex = _exact_monomial(c, h, e)
        scale = r.vol * float(np.prod((c + h) ** np.array(e)))
        assert abs(r.i7 - ex) <= 1e-13 * scale, (e, r.i7, ex)
        if sum(e) <= 5:
            assert abs(r.i5 - ex) <= 1e-13 * scale, (e, r.i5, ex)


def test_weights_sum_to_one(oracle):
    for d in range(1, 13):
        r = oracle.rule(np.full(d, 0.5), np.full(d, 0.25), f=lambda x: 1.0)
        assert abs(r.i7 - r.vol) <= 1e-14 * r.vol
        assert abs(r.i5 - r.vol) <= 1e-14 * r.vol
        assert r.err <= 1e-14 * r.vol


def test_d1_moment_equations(oracle):
    """For d = 1 the rule has nodes 0, +-l2, +-l3, +-l5 (class 4 is empty);
    its four weights are the unique solution of the moment equations on
    [-1, 1] for 1, x^2, x^4, x^6.  The embedded rule uses 0, +-l2, +-l3 and
    is fixed by the moments 1, x^2, x^4."""
    nodes = []
    oracle.rule([0.0], [1.0], f=lambda x: nodes.append(float(x[0])) or 0.0)
    pos = sorted({abs(v) for v in nodes if v != 0.0})
    assert len(nodes) == 7 and len(pos) == 3
    # weights of the 7-point rule from the moments
    t = np.array([0.0] + pos)
    A = np.array([[1.0 if p == 0 else 0.0] + [2 * t[i] ** (2 * p) for i in range(1, 4)]
                  for p in range(4)])
    b = np.array([2.0 / (2 * p + 1) for p in range(4)])
    W7 = np.linalg.solve(A, b)
    for f in (math.exp, math.cos, lambda x: 1.0 / (2.0 + x), lambda x: x ** 7 + 3 * x ** 6):
        r = oracle.rule([0.0], [1.0], f=lambda x, f=f: f(float(x[0])))
        ref = W7[0] * f(0.0) + sum(W7[i] * (f(t[i]) + f(-t[i])) for i in range(1, 4))
        assert abs(r.i7 - ref) <= 2e-15 * max(1.0, abs(ref))
    # the embedded degree-5 rule lives on exactly two of the three radii:
    # exactly one choice of dropped radius reproduces I5 for every f, and it
    # is the middle radius (the sign-class generator sqrt(9/19))
    matches = []
    for drop in range(1, 4):
        tt = [t[i] for i in range(1, 4) if i != drop]
        A5 = np.array([[1.0 if p == 0 else 0.0] + [2 * v ** (2 * p) for v in tt]
                       for p in range(3)])
        W5 = np.linalg.solve(A5, b[:3])
        ok = True
        for f in (math.exp, math.cos, lambda x: 1.0 / (2.0 + x)):
            r = oracle.rule([0.0], [1.0], f=lambda x, f=f: f(float(x[0])))
            ref5 = W5[0] * f(0.0) + sum(w * (f(v) + f(-v)) for w, v in zip(W5[1:], tt))
            ok = ok and abs(r.i5 - ref5) <= 4e-15
        if ok:
            matches.append(drop)
    assert matches == [2]


def test_symmetry_permutation_and_reflection(oracle):
    rng = random.Random(7)
    d = 5
    c, h = _box(rng, d)
    a = np.array([rng.uniform(0.5, 2) for _ in range(d)])

    def f(x):
        return math.exp(-float(np.sum(a * (x - 0.3) ** 2))) + 0.1 * x[0] * x[3] ** 3

    base = oracle.rule(c, h, f=f)
    perm = [3, 1, 4, 0, 2]
    inv = np.argsort(perm)

    def fp(y):  # y is the permuted coordinate vector
        return f(y[inv])

    rp = oracle.rule(c[perm], h[perm], f=fp)
    assert abs(rp.i7 - base.i7) <= 1e-14 * abs(base.i7)
    assert abs(rp.i5 - base.i5) <= 1e-14 * abs(base.i5)
    assert np.allclose(rp.D, base.D[perm], rtol=1e-10, atol=1e-15)
    # reflection about the centre: f(2c - x)
    rr = oracle.rule(c, h, f=lambda x: f(2 * c - x))
    assert abs(rr.i7 - base.i7) <= 1e-13 * abs(base.i7)
    assert abs(rr.i5 - base.i5) <= 1e-13 * abs(base.i5)
    assert np.allclose(rr.D, base.D, rtol=1e-9, atol=1e-15)


def test_class_sums_of_symmetric_function(oracle):
    """For a permutation-symmetric f on a cube the class sums are invariant
    under any relabelling of axes, and each class sum is its size times the
    common value when f depends only on the multiset of |x_k - c_k|."""
    d = 4
    c = np.full(d, 0.5)
    h = np.full(d, 0.25)
    g = lambda x: math.exp(-float(np.sum((x - 0.5) ** 2)))
    r = oracle.rule(c, h, f=g)
    lam = oracle.lambdas()
    v2 = math.exp(-(lam[0] * 0.25) ** 2)
    v3 = math.exp(-(lam[1] * 0.25) ** 2)
    v4 = math.exp(-2 * (lam[2] * 0.25) ** 2)
    v5 = math.exp(-d * (lam[3] * 0.25) ** 2)
    assert abs(r.s[0] - 1.0) < 1e-15
    assert abs(r.s[1] - 2 * d * v2) < 1e-13
    assert abs(r.s[2] - 2 * d * v3) < 1e-13
    assert abs(r.s[3] - 2 * d * (d - 1) * v4) < 1e-13
    assert abs(r.s[4] - 2 ** d * v5) < 1e-13


def test_odd_about_centre_integrates_to_zero(oracle):
    rng = random.Random(11)
    d = 3
    c, h = _box(rng, d)
    f = lambda x: (x[0] - c[0]) ** 3 * (x[1] - c[1]) ** 2 + (x[2] - c[2])
    r = oracle.rule(c, h, f=f)
    assert abs(r.i7) <= 1e-15 * r.vol and abs(r.i5) <= 1e-15 * r.vol


def test_fourth_difference_properties(oracle):
    rng = random.Random(5)
    d = 4
    c, h = _box(rng, d)
    for k in range(d):
        r = oracle.rule(c, h, f=lambda x, k=k: (x[k] - 0.1) ** 4)
        others = [j for j in range(d) if j != k]
        assert r.D[k] > 1e-6 and all(r.D[j] == 0.0 for j in others)
        assert r.axis == k
    # cubics: every fourth difference is at round-off level -> flat rule
    cub = lambda x: 1.0 + x[0] ** 3 - 2 * x[1] ** 2 * x[2] + x[3]
    r = oracle.rule(c, h, f=cub)
    assert r.flat and np.all(r.D <= 1e-13)
    assert r.axis == int(np.argmax(h))
    # the axis with the strongest quartic term wins
    r = oracle.rule(np.full(d, 0.5), np.full(d, 0.5),
                    f=lambda x: x[0] ** 4 + 3 * x[2] ** 4 + 2 * x[3] ** 4)
    assert r.axis == 2
    # lowest index on exact ties
    r = oracle.rule(np.full(d, 0.5), np.full(d, 0.5), f=lambda x: x[1] ** 4 + x[3] ** 4)
    assert r.axis == 1 and r.axis_tie


def test_fourth_difference_is_a_fourth_difference(oracle):
    """D_k = |(f(+l2)+f(-l2)-2f0) - (l2/l3)^2 (f(+l3)+f(-l3)-2f0)|: for
    f = x^4 on [-1,1] this is 2 l2^2 |l2^2 - l3^2| (hand-derived)."""
    lam = oracle.lambdas()
    r = oracle.rule([0.0], [1.0], f=lambda x: float(x[0]) ** 4)
    want = 2 * lam[0] ** 2 * abs(lam[0] ** 2 - lam[1] ** 2)
    assert abs(r.D[0] - want) <= 1e-15


def test_lambda_values_from_exactness(oracle):
    """The generators are pinned by exactness in d >= 2 (mixed monomials
    x^2 y^2, x^2 y^2 z^2, x^4 y^2 ...); check them against the published
    squares 9/70, 9/10, 9/10, 9/19 (Genz & Malik 1980)."""
    lam = oracle.lambdas()
    assert np.allclose(lam ** 2, [9 / 70, 9 / 10, 9 / 10, 9 / 19], rtol=1e-15)


def test_split_guard(oracle):
    # half-widths below half an ulp of the centre: bisection cannot move the
    # centre, so the guard fires (flat differences -> widest axis, index 0)
    c = np.array([0.5, 0.5])
    h = np.array([1e-17, 1e-17])
    r = oracle.rule(c, h, f=lambda x: float(x[0]) ** 4)
    assert r.flat and r.axis == 0 and r.split_bad
    r = oracle.rule(c, np.array([0.25, 0.25]), f=lambda x: float(x[0]) ** 4)
    assert not r.split_bad


def test_near_tie_flag_stays_off_for_clear_choices(oracle):
    """The axis near-tie flag must not fire when the choice is clear: a
    parity test skips flagged axes, so a flag that over-fires would hide
    mismatches.  Fourth differences in ratio 2:1 (x_0^4 against x_1^4 / 2),
    and a clearly non-flat exponential, are not near-ties."""
    c, h = [0.4, 0.55, 0.5], [0.3, 0.3, 0.2]  # equal widths on axes 0 and 1
    r = oracle.rule(c, h, f=lambda x: x[0] ** 4 + 0.5 * x[1] ** 4 + x[2])
    assert r.axis == 0 and not r.axis_tie and not r.flat
    assert r.D[0] > 1.9 * r.D[1] and r.D[2] <= 1e-15 * r.D[0]
    r = oracle.rule(c, h, f=lambda x: math.exp(0.3 * x[0] + 2.0 * x[1] - x[2]))
    assert r.axis == 1 and not r.axis_tie
    # runner-up 1e-9 below the best (far outside the 1e-12 band): no flag;
    # 1e-14 below: flagged
    r = oracle.rule([0.5, 0.5], [0.5, 0.5], f=lambda x: x[0] ** 4 + (1 - 1e-9) * x[1] ** 4)
    assert r.axis == 0 and not r.axis_tie
    r = oracle.rule([0.5, 0.5], [0.5, 0.5], f=lambda x: x[0] ** 4 + (1 - 1e-14) * x[1] ** 4)
    assert r.axis == 0 and r.axis_tie
