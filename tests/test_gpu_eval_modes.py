"""The FP64 rule kernel's two ways of evaluating f at a region's nodes
(gmq_set_eval_mode; paper Sec. 2: the rule applies f at every node).

* node-wise (f from each node's coordinates) against the oracle per region,
  with the per-region tolerances of test_gpu_parity.py;
* both modes give every lane mapping the same bits;
* the two modes agree per region within 1e-13 of the terms' magnitude (they
  differ only in the rounding order of the inner chain S);
* end to end with node-wise evaluation, sweep by sweep against the oracle
  (tests/loop_parity.py);
* the batched form does not depend on the context's mode;
* an unknown mode is rejected.
"""
import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G
from tests.loop_parity import assert_loop_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _soa(x):
    return torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device="cuda")


def _params(fam, d, seed=3):
    if fam == G.PRODUCT_PEAK:
        return G.seed_genz(seed, fam, d, 5.0 * d)
    if fam == G.DISCONTINUOUS:
        a, u = G.seed_genz(seed, fam, d, 2.0)
        return a, 0.3 + 0.6 * u
    if fam == G.POLY_SUMSQ11:
        return np.zeros(d), np.zeros(d)
    return G.seed_genz(seed, fam, d, G.GENZ_TARGET_SUM.get(fam, 2.0))


@pytest.fixture
def nodewise(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    gpu_ctx.set_eval_mode(gmq.EVAL_NODEWISE)
    yield gpu_ctx
    gpu_ctx.set_eval_mode(gmq.EVAL_SEPARABLE)


@pytest.mark.parametrize("fam", range(7))
@pytest.mark.parametrize("d", [1, 3, 8])
@pytest.mark.parametrize("lanes", [1, 32])
def test_nodewise_per_region(oracle, nodewise, fam, d, lanes):
    a, u = _params(fam, d)
    n = {1: 1500, 3: 800, 8: 120}[d]
    c, h = G.random_boxes(50 + d, n, d)
    o = oracle.rule_regions(fam, a, u, c, h)
    i7, err, vf, ax = nodewise.eval_rule(fam, a, u, _soa(c), _soa(h), lanes=lanes)
    scale = o["i7abs"]
    assert np.all(np.abs(i7.cpu().numpy() - o["i7"]) <= 1e-12 * scale)
    assert np.all(np.abs(err.cpu().numpy() - o["err"]) <= 1e-12 * scale)
    assert np.array_equal(vf.cpu().numpy(), o["vol"])
    tie = o["axis_tie"].astype(bool)
    ax = ax.cpu().numpy().astype(np.int32)
    assert np.array_equal((ax & 0x7F)[~tie], o["axis"][~tie])
    assert np.array_equal((ax >> 7)[~tie], o["split_bad"][~tie])


@pytest.mark.parametrize("fam", [G.OSCILLATORY, G.PRODUCT_PEAK, G.CORNER_PEAK, G.GAUSSIAN,
                                 G.C0, G.DISCONTINUOUS])
@pytest.mark.parametrize("d", [2, 5, 9, 12])
def test_modes_lane_mappings_and_agreement(oracle, gpu_ctx, fam, d):
    from paper_2511_01573_gb300 import gmq
    a, u = _params(fam, d, 5)
    c, h = G.random_boxes(70 + d, {2: 700, 5: 200, 9: 40, 12: 9}[d], d)
    cd, hd = _soa(c), _soa(h)
    res = {}
    try:
        for mode in (gmq.EVAL_SEPARABLE, gmq.EVAL_NODEWISE):
            gpu_ctx.set_eval_mode(mode)
            outs = [gpu_ctx.eval_rule(fam, a, u, cd, hd, lanes=t) for t in (1, 4, 32, 128)]
            for o in outs[1:]:
                for x, y in zip(outs[0], o):
                    assert torch.equal(x, y), (mode, fam, d)
            res[mode] = [x.cpu().numpy() for x in outs[0]]
    finally:
        gpu_ctx.set_eval_mode(gmq.EVAL_SEPARABLE)
    scale = oracle.rule_regions(fam, a, u, c, h)["i7abs"]
    s, nw = res[gmq.EVAL_SEPARABLE], res[gmq.EVAL_NODEWISE]
    assert np.all(np.abs(s[0] - nw[0]) <= 1e-13 * scale)
    assert np.all(np.abs(s[1] - nw[1]) <= 1e-13 * scale)
    assert np.array_equal(s[2], nw[2])


@pytest.mark.parametrize("fam,d,tol", [(G.C0, 4, 1e-6), (G.CORNER_PEAK, 8, 1e-4),
                                       (G.GAUSSIAN, 5, 1e-9)])
def test_nodewise_end_to_end(oracle, nodewise, fam, d, tol):
    a, u = _params(fam, d, seed=2)
    o = oracle.integrate(fam, a, u, tol, max_regions=1 << 22)
    g = nodewise.integrate(fam, a, u, tol, max_regions=1 << 22)
    assert o.status == g.status == 0
    assert_loop_parity(o, g, nodewise.last_trace())


def test_batch_does_not_depend_on_the_mode(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    probs = [G.Problem(fam, d, *_params(fam, d, seed=4), 1e-6)
             for fam, d in ((G.C0, 3), (G.GAUSSIAN, 5), (G.CORNER_PEAK, 4))]
    ref = gpu_ctx.integrate_batch(probs, max_regions=1 << 20)
    try:
        gpu_ctx.set_eval_mode(gmq.EVAL_NODEWISE)
        got = gpu_ctx.integrate_batch(probs, max_regions=1 << 20)
    finally:
        gpu_ctx.set_eval_mode(gmq.EVAL_SEPARABLE)
    for r, s in zip(ref, got):
        assert (r.integral, r.error, r.regions_evaluated) == (s.integral, s.error,
                                                              s.regions_evaluated)
    for p, r in zip(probs, ref):
        s = gpu_ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=1 << 20)
        assert (r.integral, r.regions_evaluated) == (s.integral, s.regions_evaluated)


def test_unknown_mode_rejected(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    with pytest.raises(gmq.GmqError):
        gpu_ctx.set_eval_mode(2)


@pytest.mark.parametrize("fam", range(7))
@pytest.mark.parametrize("d", [1, 2, 4, 6, 9, 12])
def test_adjoint_modes_agree(oracle, gpu_ctx, fam, d):
    """gmq_rule_grad: the separable per-row sums against the node-wise
    derivatives and against the oracle on random boxes (1e-12 of the largest
    component, as the adjoint tests hold the node-wise kernel)."""
    from paper_2511_01573_gb300 import gmq
    a, u = G.seed_uniform(13 + d, fam, d, 0.5, 3.0)
    if fam == G.DISCONTINUOUS:
        u = 0.3 + 0.6 * u
    c, h = G.random_boxes(90 + d, {1: 400, 2: 300, 4: 120, 6: 60, 9: 12, 12: 4}[d], d)
    go, qo = oracle.rule_grad(fam, a, u, c, h)
    res = {}
    try:
        for mode in (gmq.EVAL_SEPARABLE, gmq.EVAL_NODEWISE):
            gpu_ctx.set_eval_mode(mode)
            res[mode] = gpu_ctx.rule_grad(fam, a, u, _soa(c), _soa(h))
    finally:
        gpu_ctx.set_eval_mode(gmq.EVAL_SEPARABLE)
    scale = np.max(np.abs(go)) + abs(qo)
    for mode, (g, q) in res.items():
        assert abs(q - qo) <= 1e-12 * max(abs(qo), scale), (mode, q, qo)
        assert np.all(np.abs(np.asarray(g) - go) <= 1e-12 * scale), (mode, g, go)
