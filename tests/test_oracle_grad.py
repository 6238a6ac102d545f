"""Pins of the oracle's frozen-partition gradient (the adjoint extension;
no counterpart in the paper).

Q(theta) = sum over the final partition of the degree-7 rule value; its
gradient is the same rule applied to df/dtheta.  Pinned by
* central finite differences of Q itself (h = 1e-5) on the same partition;
* the closed-form gradient of the Gaussian family's exact integral
  (product of erf factors), to within the integration tolerance;
* the recorded partition tiles the domain and reproduces the integral.
"""
import math

import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G


def _fd(oracle, fam, a, u, c, h, step=1e-5):
    d = len(a)
    out = np.zeros(2 * d)
    for k in range(2 * d):
        da = np.zeros(d)
        du = np.zeros(d)
        (da if k < d else du)[k % d] = step
        _, qp = oracle.rule_grad(fam, a + da, u + du, c, h)
        _, qm = oracle.rule_grad(fam, a - da, u - du, c, h)
        out[k] = (qp - qm) / (2 * step)
    return out


@pytest.mark.parametrize("fam", [G.OSCILLATORY, G.PRODUCT_PEAK, G.CORNER_PEAK, G.GAUSSIAN, G.C0])
def test_gradient_matches_finite_differences(oracle, fam):
    d = 3
    a, u = G.seed_uniform(7, fam, d, 0.5, 3.0)
    r, c, h = oracle.integrate_partition(fam, a, u, 1e-6, max_regions=1 << 18)
    assert r.status == 0 and c is not None
    g, q = oracle.rule_grad(fam, a, u, c, h)
    fd = _fd(oracle, fam, a, u, c, h)
    scale = np.max(np.abs(g))
    # C0's u-derivative jumps where a node sits on the kink x_j = u_j: a
    # finite difference across it is no check, so only its a-part is compared
    k = d if fam == G.C0 else 2 * d
    assert np.all(np.abs(fd[:k] - g[:k]) <= 1e-7 * scale), (fd, g)
    if fam == G.CORNER_PEAK:
        assert np.all(g[d:] == 0.0)  # no u-dependence
    if fam == G.OSCILLATORY:
        assert np.all(g[d + 1:] == 0.0)  # only u_1 enters


def test_partition_tiles_domain_and_reproduces_integral(oracle):
    a, u = G.seed_uniform(3, G.GAUSSIAN, 4, 0.5, 3.0)
    r, c, h = oracle.integrate_partition(G.GAUSSIAN, a, u, 1e-8, max_regions=1 << 20)
    assert r.status == 0
    assert abs(np.prod(2 * h, axis=1).sum() - 1.0) < 1e-13
    _, q = oracle.rule_grad(G.GAUSSIAN, a, u, c, h)
    assert abs(q - r.integral) <= 1e-13 * abs(r.integral)


def _gauss_closed_grad(a, u):
    g = np.array([math.sqrt(math.pi) / (2 * ai) * (math.erf(ai * (1 - ui)) + math.erf(ai * ui))
                  for ai, ui in zip(a, u)])
    dga = np.array([-gi / ai + ((1 - ui) * math.exp(-(ai * (1 - ui)) ** 2)
                                + ui * math.exp(-(ai * ui) ** 2)) / ai
                    for gi, ai, ui in zip(g, a, u)])
    dgu = np.array([math.exp(-(ai * ui) ** 2) - math.exp(-(ai * (1 - ui)) ** 2)
                    for ai, ui in zip(a, u)])
    I = float(np.prod(g))
    return I, np.concatenate([I / g * dga, I / g * dgu])


def test_gaussian_gradient_against_closed_form(oracle):
    for seed in (1, 2, 3):
        a, u = G.seed_uniform(seed, G.GAUSSIAN, 3, 0.5, 3.0)
        r, c, h = oracle.integrate_partition(G.GAUSSIAN, a, u, 1e-8, max_regions=1 << 20)
        g, q = oracle.rule_grad(G.GAUSSIAN, a, u, c, h)
        I, gex = _gauss_closed_grad(a, u)
        assert abs(q - I) <= 1e-7 * I
        assert np.all(np.abs(g - gex) <= 1e-6 * np.max(np.abs(gex))), (g, gex)
