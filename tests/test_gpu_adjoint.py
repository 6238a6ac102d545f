"""Adjoint (gradient) extension on the GPU against the oracle.

* the run matches the oracle's sweep by sweep (tests/loop_parity.py), and
  the final partition the GPU records equals the oracle's (same regions in
  the same order) when no decision of the run is a flagged near-tie;
* gmq_rule_grad on a partition equals the oracle's or_rule_grad on the same
  partition (FP64, 1e-12 of the largest component);
* it is the derivative of the frozen-partition quadrature: central
  differences (h = 1e-5) of the GPU's own quadrature sum on that partition;
* on converged partitions of the d = 6 Gaussian family with a_j ~ U(0.5, 3),
  u_j ~ U(0, 1) at tol 1e-8 it matches the closed-form erf-product gradient;
* the torch.autograd.Function returns the same numbers.
"""
import math

import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G
from tests.loop_parity import assert_loop_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _np(t):
    return t.detach().cpu().numpy().T.copy()


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


@pytest.mark.parametrize("fam,d,tol", [(G.GAUSSIAN, 3, 1e-7), (G.C0, 3, 1e-5),
                                       (G.OSCILLATORY, 4, 1e-6), (G.PRODUCT_PEAK, 2, 1e-7),
                                       (G.CORNER_PEAK, 4, 1e-6)])
def test_partition_and_gradient_match_oracle(oracle, gpu_ctx, fam, d, tol):
    a, u = G.seed_uniform(11, fam, d, 0.5, 3.0)
    r = gpu_ctx.integrate(fam, a, u, tol, max_regions=1 << 20, keep_partition=True)
    c, h = gpu_ctx.partition_copy()
    assert r.status == 0
    # the leaves tile the unit cube
    vol = torch.prod(2 * h, dim=0).sum().item()
    assert abs(vol - 1.0) < 1e-12
    ro, co, ho = oracle.integrate_partition(fam, a, u, tol, max_regions=1 << 20)
    o = oracle.integrate(fam, a, u, tol, max_regions=1 << 20)
    k = assert_loop_parity(o, r, gpu_ctx.last_trace())
    if k == len(o.trace):
        # no flagged decision anywhere: the same leaves in the same order
        assert np.array_equal(_np(c), co) and np.array_equal(_np(h), ho)
    else:
        # a flagged axis or classification may change which leaves exist;
        # both partitions still tile the domain
        assert abs(np.prod(2 * ho, axis=1).sum() - 1.0) < 1e-12
    g, q = gpu_ctx.rule_grad(fam, a, u, c, h)
    go, qo = oracle.rule_grad(fam, a, u, _np(c), _np(h))
    scale = np.max(np.abs(go)) + abs(qo)
    assert abs(q - qo) <= 1e-12 * abs(qo)
    assert np.all(np.abs(g - go) <= 1e-12 * scale), (g, go)
    assert abs(q - r.integral) <= 1e-12 * abs(r.integral)


@pytest.mark.parametrize("fam", [G.GAUSSIAN, G.OSCILLATORY, G.PRODUCT_PEAK, G.CORNER_PEAK])
def test_gradient_is_derivative_of_frozen_quadrature(gpu_ctx, fam):
    d = 4
    a, u = G.seed_uniform(5, fam, d, 0.5, 3.0)
    gpu_ctx.integrate(fam, a, u, 1e-7, max_regions=1 << 20, keep_partition=True)
    c, h = gpu_ctx.partition_copy()
    g, q = gpu_ctx.rule_grad(fam, a, u, c, h)
    step = 1e-5
    for k in range(2 * d):
        da = np.zeros(d)
        du = np.zeros(d)
        (da if k < d else du)[k % d] = step
        i7p, _, _, _ = gpu_ctx.eval_rule(fam, a + da, u + du, c, h)
        i7m, _, _, _ = gpu_ctx.eval_rule(fam, a - da, u - du, c, h)
        fd = (gpu_ctx.tree_sum(i7p) - gpu_ctx.tree_sum(i7m)) / (2 * step)
        assert abs(fd - g[k]) <= 1e-7 * np.max(np.abs(g)), (k, fd, g[k])


def test_gaussian_d6_gradients_against_closed_form(gpu_ctx):
    # the first parameter sets of the 1024-set d = 6 workload; sharp
    # Gaussians (a_j up to 3) need ~10^7 regions at 1e-8, hence the 2^24 pool
    sets = G.gaussian_grad_sets(count=1024, dim=6)
    for a, u in sets[:6]:
        r = gpu_ctx.integrate(G.GAUSSIAN, a, u, 1e-8, max_regions=1 << 24, keep_partition=True)
        assert r.status == 0
        c, h = gpu_ctx.partition_copy()
        g, q = gpu_ctx.rule_grad(G.GAUSSIAN, a, u, c, h)
        I, gex = _gauss_closed_grad(a, u)
        assert abs(q - I) <= 1e-7 * I
        assert np.all(np.abs(g - gex) <= 1e-6 * np.max(np.abs(gex))), (g, gex)


def test_autograd_function(gpu_ctx):
    from paper_2511_01573_gb300 import autograd as AG
    a0, u0 = G.seed_uniform(3, G.GAUSSIAN, 5, 0.5, 3.0)
    a = torch.tensor(a0, requires_grad=True)
    u = torch.tensor(u0, requires_grad=True)
    I = AG.integral(a, u, rel_tol=1e-8, context=gpu_ctx)
    I.backward()
    c, h = gpu_ctx.partition_copy()
    g, q = gpu_ctx.rule_grad(G.GAUSSIAN, a0, u0, c, h)
    assert I.item() == pytest.approx(q, rel=1e-12)
    assert np.allclose(a.grad.numpy(), g[:5], rtol=1e-12, atol=0)
    assert np.allclose(u.grad.numpy(), g[5:], rtol=1e-12, atol=0)
    # batched rows with an upstream weight per row
    A = torch.tensor(np.stack([a0, a0 * 1.1]), requires_grad=True)
    U = torch.tensor(np.stack([u0, u0]), requires_grad=True)
    out = AG.integral(A, U, rel_tol=1e-8, context=gpu_ctx)
    (out * torch.tensor([1.0, -2.0], dtype=torch.float64)).sum().backward()
    assert np.allclose(A.grad[0].numpy(), g[:5], rtol=1e-12)
    I2, gex2 = _gauss_closed_grad(a0 * 1.1, u0)
    assert np.allclose(A.grad[1].numpy(), -2.0 * gex2[:5], rtol=1e-5)


def test_partition_keep_flags(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    a, u = G.seed_genz(1, G.C0, 3, 2.0)
    gpu_ctx.integrate(G.C0, a, u, 1e-5, keep_partition=False)
    with pytest.raises(RuntimeError):
        gpu_ctx.partition_copy()
    # a run stopped by the sweep limit still leaves a valid partition
    r = gpu_ctx.integrate(G.C0, a, u, 1e-9, max_iters=4, keep_partition=True)
    assert r.status == gmq.MAX_ITERS
    c, h = gpu_ctx.partition_copy()
    assert abs(torch.prod(2 * h, dim=0).sum().item() - 1.0) < 1e-12
    assert gmq.pool_bytes(3, 1 << 20, gmq.KEEP_PARTITION) > gmq.pool_bytes(3, 1 << 20)
