"""Pins of the oracle's tensor-product Gauss-Kronrod (7, 15) rule against
mathematics, not against itself.

* The 1-D tables: the Gauss part equals numpy's Gauss-Legendre routine; the
  15-point rule integrates every polynomial of degree <= 22 exactly (a
  15-point rule that contains the 7 Gauss nodes and has degree 22 is
  Kronrod's extension, so this identifies it) and fails at degree 24; the
  Gauss part is exact to degree 13 and fails at 14; nodes symmetric and
  interlacing, weights positive.
* The tensor rule on boxes: exact for products of monomials of degree <= 22
  per axis (K) and <= 13 (G); the directional estimates vanish along axes
  on which the integrand is constant and pick the axis that carries the
  error; reflection symmetry; the flat fallback.
* The adaptive loop with the rule reaches closed forms.
"""
import math

import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G
from tests import closed_forms as CF


def test_gauss_part_is_gauss_legendre(oracle):
    t = oracle.gk_table()
    x, wk, wg = t[:15], t[15:30], t[30:]
    gi = [i for i in range(15) if wg[i] != 0.0]
    assert gi == list(range(1, 15, 2))
    g, w = np.polynomial.legendre.leggauss(7)
    assert np.allclose(x[gi], g, rtol=0, atol=4e-16)
    assert np.allclose(wg[gi], w, rtol=0, atol=4e-16)


def test_kronrod_exactness_and_structure(oracle):
    t = oracle.gk_table()
    x, wk, wg = t[:15], t[15:30], t[30:]
    assert np.all(np.diff(x) > 0) and np.array_equal(x, -x[::-1])
    assert np.array_equal(wk, wk[::-1]) and np.all(wk > 0)
    for p in range(0, 26):
        exact = 2.0 / (p + 1) if p % 2 == 0 else 0.0
        k = float(np.dot(wk, x ** p))
        gq = float(np.dot(wg, x ** p))
        if p <= 22:
            assert abs(k - exact) <= 2e-16 * 8, p
        elif p == 24:
            assert abs(k - exact) > 1e-10
        if p <= 13:
            assert abs(gq - exact) <= 2e-16 * 8, p
        elif p == 14:
            assert abs(gq - exact) > 1e-6
    # Kronrod-only nodes interlace the Gauss nodes (alternate in the sorted list)
    assert all((wg[i] == 0.0) == (i % 2 == 0) for i in range(15))


def _box_monomial(c, h, m):
    """Exact integral of prod x_k^{m_k} over the box c +- h."""
    v = 1.0
    for ck, hk, mk in zip(c, h, m):
        lo, hi = ck - hk, ck + hk
        v *= (hi ** (mk + 1) - lo ** (mk + 1)) / (mk + 1)
    return v


@pytest.mark.parametrize("m", [(0, 0, 0), (22, 0, 5), (13, 13, 13), (7, 22, 1), (20, 21, 22)])
def test_tensor_rule_exact_per_axis_degree(oracle, m):
    c, h = [0.3, -0.2, 0.55], [0.25, 0.4, 0.1]
    f = lambda x: float(np.prod(x ** np.array(m)))
    r, _ = oracle.rule_gk(c, h, f=f)
    ex = _box_monomial(c, h, m)
    assert abs(r["ik"] - ex) <= 1e-13 * max(1.0, abs(ex))
    if max(m) <= 13:
        assert abs(r["ig"] - ex) <= 1e-13 * max(1.0, abs(ex))
    assert r["vol"] == pytest.approx(np.prod(2 * np.array(h)), rel=0, abs=0)


def test_directional_estimates_find_the_axis(oracle):
    c, h = [0.5, 0.5, 0.5, 0.5], [0.5, 0.5, 0.5, 0.5]
    # degree 14 along axis 2 only: G7 is inexact there, exact elsewhere
    r, E = oracle.rule_gk(c, h, f=lambda x: x[2] ** 14 + 3.0)
    assert r["axis"] == 2 and not r["flat"]
    assert E[2] > 1e-10 * r["scale"]
    assert np.all(np.delete(E, 2) <= 1e-14 * r["scale"])
    assert r["err"] == pytest.approx(E[2], rel=1e-12)
    # two inexact axes: the larger directional error wins
    r, E = oracle.rule_gk(c, h, f=lambda x: x[1] ** 14 + 2.0 * x[3] ** 14)
    assert r["axis"] == 3 and E[3] > E[1] > 0


def test_flat_fallback_and_reflection(oracle):
    c, h = [0.5, 0.4, 0.6], [0.2, 0.3, 0.1]
    r, E = oracle.rule_gk(c, h, f=lambda x: 1.0 + x[0] - 2 * x[1] * x[2])
    assert r["flat"] and r["axis"] == 1  # widest half-width
    f = lambda x: math.exp(-(x[0] - 0.3) ** 2 - 2 * (x[1] - 0.1) ** 2) * (1 + x[2])
    g = lambda x: f(2 * np.array(c) - x)
    r1, _ = oracle.rule_gk(c, h, f=f)
    r2, _ = oracle.rule_gk(c, h, f=g)
    assert r1["ik"] == pytest.approx(r2["ik"], rel=1e-14)
    assert r1["ig"] == pytest.approx(r2["ig"], rel=1e-14)


def test_regions_call_matches_single(oracle):
    a, u = G.seed_genz(4, G.C0, 3, 2.0)
    c, h = G.random_boxes(5, 6, 3)
    o = oracle.rule_gk_regions(G.C0, a, u, c, h)
    for r in range(6):
        s, _ = oracle.rule_gk(c[r], h[r], family=G.C0, a=a, u=u)
        assert o["ik"][r] == s["ik"] and o["err"][r] == s["err"] and o["axis"][r] == s["axis"]


@pytest.mark.parametrize("fam,d,tol", [(G.GAUSSIAN, 3, 1e-10), (G.PRODUCT_PEAK, 2, 1e-9),
                                       (G.C0, 2, 1e-7), (G.OSCILLATORY, 4, 1e-8)])
def test_gk_loop_reaches_closed_forms(oracle, fam, d, tol):
    a, u = G.seed_genz(7, fam, d, G.GENZ_TARGET_SUM.get(fam, 5.0 * d))
    res = oracle.integrate(fam, a, u, tol, max_regions=1 << 16, rule=oracle.RULE_GK)
    ex = CF.exact(fam, a, u)
    assert res.status == 0
    assert abs(res.integral - ex) <= 10 * tol * abs(ex)
    assert res.function_evals == res.regions_evaluated * 15 ** d


def test_gk_dimension_limit(oracle):
    a, u = G.seed_genz(1, G.GAUSSIAN, 7, 3.5)
    assert oracle.integrate(G.GAUSSIAN, a, u, 1e-3, rule=oracle.RULE_GK).status == -1
