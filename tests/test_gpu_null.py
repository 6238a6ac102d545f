"""The null-rule error estimate (GMQ_EST_NULL_RULES; paper Sec. 2 cites the
Berntsen-Espelid-Genz heuristic) on the GPU against the oracle.

* per region (FP64): I7 as for the embedded estimate; the estimate within
  the oracle's rounding band of its own value (the band bounds how far
  class sums added in another order can move it, and includes the other
  regime's value where that band reaches across r = 1); the library's
  null-rule table against the oracle's exact one;
* every lane mapping gives the same bits;
* end to end, sweep by sweep against the oracle's run with the same
  estimator (tests/loop_parity.py), and the batched form bit-identical to
  single runs;
* the mixed form with null rules meets the tolerance against closed forms.
"""
import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G
from tests import closed_forms as CF
from tests.loop_parity import assert_loop_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NULL = 1


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


def test_library_table_matches_the_oracles(oracle):
    """The library builds its table in FP64 on the host by another route
    (orthogonalised moment functionals; the host compiler may fuse its
    multiply-adds), the oracle in exact rationals: they agree to 1e-13 of
    the largest weight."""
    from paper_2511_01573_gb300 import gmq
    for d in (1, 2, 3, 4, 5, 8, 12, 16):
        lib, ref = gmq.null_rule_table(d), oracle.null_table(d).reshape(4, 5)
        n = np.array([1, 2 * d, 2 * d, 2 * d * (d - 1), 2.0 ** d])
        for k in (0, 3):  # unique up to sign
            s = np.sign(np.sum(n * lib[k] * ref[k]))
            assert np.max(np.abs(s * lib[k] - ref[k])) <= 1e-13 * np.max(np.abs(ref[k]))
        # rows 2, 3 span the same plane: the sum of their outer products does
        # not depend on the basis chosen in it
        pl, pr = lib[1:3].T @ lib[1:3], ref[1:3].T @ ref[1:3]
        assert np.max(np.abs(pl - pr)) <= 1e-13 * np.max(np.abs(pr))


@pytest.mark.parametrize("fam", range(7))
@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_null_estimate_per_region(oracle, gpu_ctx, fam, d):
    a, u = _params(fam, d)
    n = {1: 1500, 2: 1200, 3: 800, 5: 300, 8: 100}[d]
    c, h = G.random_boxes(40 + d, n, d)
    # the random boxes and boxes 1/50 their size (resolved, asymptotic)
    c = np.concatenate([c, c])
    h = np.concatenate([h, h / 50.0])
    o = oracle.rule_regions_est(fam, a, u, c, h)
    for lanes in (1, 32):
        i7, err, _, ax = gpu_ctx.eval_rule(fam, a, u, _soa(c), _soa(h), lanes=lanes,
                                           estimator=NULL)
        i7, err = i7.cpu().numpy(), err.cpu().numpy()
        assert np.all(np.abs(i7 - o["i7"]) <= 1e-12 * o["scale"])
        # err_band: the spread of the estimate when the class sums move by
        # 1e-13 of their magnitude; the comparison allows ten times that
        bad = np.abs(err - o["err"]) > 10.0 * o["err_band"]
        assert not bad.any(), (fam, d, lanes, np.nonzero(bad)[0][:5], err[bad][:3], o["err"][bad][:3])
        tie = o["axis_tie"].astype(bool)
        assert np.array_equal((ax.cpu().numpy() & 0x7F)[~tie], o["axis"][~tie])


@pytest.mark.parametrize("d", [4, 12])
def test_null_estimate_lane_mappings_bit_identical(gpu_ctx, d):
    a, u = _params(G.GAUSSIAN, d, 5)
    c, h = G.random_boxes(7 + d, 307 if d == 4 else 13, d)
    outs = [gpu_ctx.eval_rule(G.GAUSSIAN, a, u, _soa(c), _soa(h), lanes=t, estimator=NULL)
            for t in (1, 4, 32, 128)]
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert torch.equal(x, y)


CASES = [(G.C0, 4, 1e-6), (G.GAUSSIAN, 5, 1e-9), (G.OSCILLATORY, 6, 1e-8),
         (G.CORNER_PEAK, 5, 1e-9), (G.PRODUCT_PEAK, 3, 1e-9), (G.DISCONTINUOUS, 3, 1e-5),
         (G.C0, 8, 1e-5), (G.CORNER_PEAK, 8, 1e-7)]


@pytest.mark.parametrize("fam,d,tol", CASES)
def test_null_estimate_end_to_end(oracle, gpu_ctx, fam, d, tol):
    a, u = _params(fam, d, seed=2)
    o = oracle.integrate(fam, a, u, tol, max_regions=1 << 22, estimator=NULL)
    g = gpu_ctx.integrate(fam, a, u, tol, max_regions=1 << 22, estimator=NULL)
    assert o.status == g.status == 0
    assert_loop_parity(o, g, gpu_ctx.last_trace())


def test_null_estimate_batched_equals_single_runs(gpu_ctx):
    probs = []
    for i, (fam, d, tol) in enumerate(CASES[:6]):
        a, u = _params(fam, d, seed=2)
        probs.append(G.Problem(fam, d, a, u, tol))
    res = gpu_ctx.integrate_batch(probs, max_regions=1 << 22, estimator=NULL)
    for p, r in zip(probs, res):
        s = gpu_ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=1 << 22,
                              estimator=NULL)
        assert (r.integral, r.error, r.regions_evaluated, r.status) == (
            s.integral, s.error, s.regions_evaluated, s.status)


@pytest.mark.parametrize("fam", [G.GAUSSIAN, G.CORNER_PEAK, G.OSCILLATORY])
def test_mixed_form_with_null_rules(gpu_ctx, fam):
    from paper_2511_01573_gb300 import gmq
    d, tol = 8, 1e-5
    a, u = G.seed_genz(1, fam, d, G.GENZ_TARGET_SUM[fam])
    r = gpu_ctx.integrate(fam, a, u, tol, max_regions=1 << 22, precision=gmq.MIXED,
                          estimator=NULL)
    ex = CF.exact(fam, a, u)
    assert r.status == 0 and abs(r.integral - ex) <= tol * abs(ex)


def test_null_estimate_rejected_with_gauss_kronrod(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    a, u = G.seed_genz(1, G.GAUSSIAN, 2, 3.5)
    with pytest.raises(gmq.GmqError):
        gpu_ctx.integrate(G.GAUSSIAN, a, u, 1e-6, rule=gmq.RULE_GAUSS_KRONROD, estimator=NULL)
    c, h = G.random_boxes(1, 4, 2)
    with pytest.raises(gmq.GmqError):
        gpu_ctx.eval_rule(G.GAUSSIAN, a, u, _soa(c), _soa(h), estimator=2)
