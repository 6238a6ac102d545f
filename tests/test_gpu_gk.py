"""GPU parity of the tensor-product Gauss-Kronrod rule (gmq_eval_rule_gk and
gmq_integrate with GMQ_RULE_GAUSS_KRONROD) against the CPU oracle.

Tolerances as for the Genz-Malik path: per region |dI_K|, |d eps| <= 1e-12
of the terms' magnitude (prod h sum |wK f|; the kernel sums the 15^d terms
in another order than the oracle's node order); volume fractions, split
axes outside the oracle's near-tie flag and the guard bit bit-exact; end to
end the same sweeps, region counts and status when the oracle reports no
near-tie decision, integral within 1e-12.  The library's 1-D tables (host
FP64 Newton iteration and bisection) agree with the oracle's (exact
rational arithmetic, rounded) to 2e-14 relative.
"""
import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G
from tests import closed_forms as CF

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


def test_library_tables_match_oracle(oracle):
    from paper_2511_01573_gb300 import gmq
    lib_t = gmq.gk_table()
    ora_t = oracle.gk_table()
    # the host computation evaluates the Stieltjes polynomial in FP64 near
    # its zeros: nodes and weights within 2e-14 of the exact values
    assert np.all(np.abs(lib_t - ora_t) <= 2e-14 * np.abs(ora_t))
    assert np.array_equal(lib_t[30:] == 0.0, ora_t[30:] == 0.0)


@pytest.mark.parametrize("fam", range(7))
@pytest.mark.parametrize("d,n", [(1, 300), (2, 200), (3, 60), (4, 12)])
def test_gk_rule_per_region(oracle, gpu_ctx, fam, d, n):
    a, u = _params(fam, d)
    c, h = G.random_boxes(20 + d, n, d)
    o = oracle.rule_gk_regions(fam, a, u, c, h)
    ik, err, vf, ax = gpu_ctx.eval_rule_gk(fam, a, u, _soa(c), _soa(h))
    ik, err, vf = ik.cpu().numpy(), err.cpu().numpy(), vf.cpu().numpy()
    ax = ax.cpu().numpy().astype(np.int32)
    scale = o["scale"]
    assert np.all(np.abs(ik - o["ik"]) <= 1e-12 * scale + 1e-300), (fam, d)
    assert np.all(np.abs(err - o["err"]) <= 1e-12 * scale + 1e-300), (fam, d)
    assert np.array_equal(vf, o["vol"])
    tie = o["axis_tie"].astype(bool)
    assert np.array_equal((ax & 0x7F)[~tie], o["axis"][~tie]), (fam, d)
    assert np.array_equal((ax >> 7)[~tie], o["split_bad"][~tie])


@pytest.mark.parametrize("d", [5, 6])
def test_gk_rule_high_dimension(oracle, gpu_ctx, d):
    fam = G.GAUSSIAN
    a, u = _params(fam, d)
    c, h = G.random_boxes(40 + d, 1, d)
    o = oracle.rule_gk_regions(fam, a, u, c, h)
    ik, err, vf, ax = gpu_ctx.eval_rule_gk(fam, a, u, _soa(c), _soa(h))
    assert abs(ik.item() - o["ik"][0]) <= 1e-12 * o["scale"][0]
    assert abs(err.item() - o["err"][0]) <= 1e-12 * o["scale"][0]
    if not o["axis_tie"][0]:
        assert (int(ax.item()) & 0x7F) == o["axis"][0]


def test_gk_rule_ragged_and_limits(oracle, gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    for n in (1, 3, 4, 5, 7, 9):  # four regions per block: ragged last block
        a, u = _params(G.C0, 2)
        c, h = G.random_boxes(n, n, 2)
        o = oracle.rule_gk_regions(G.C0, a, u, c, h)
        ik, err, _, _ = gpu_ctx.eval_rule_gk(G.C0, a, u, _soa(c), _soa(h))
        assert np.all(np.abs(ik.cpu().numpy() - o["ik"]) <= 1e-12 * o["scale"])
    a, u = _params(G.GAUSSIAN, 7)
    c, h = G.random_boxes(1, 2, 7)
    with pytest.raises(gmq.GmqError):
        gpu_ctx.eval_rule_gk(G.GAUSSIAN, a, u, _soa(c), _soa(h))
    with pytest.raises(gmq.GmqError):
        gpu_ctx.integrate(G.GAUSSIAN, a, u, 1e-3, rule=gmq.RULE_GAUSS_KRONROD)
    a, u = _params(G.GAUSSIAN, 3)
    with pytest.raises(gmq.GmqError):
        gpu_ctx.integrate(G.GAUSSIAN, a, u, 1e-3, rule=gmq.RULE_GAUSS_KRONROD,
                          precision=gmq.MIXED)


@pytest.mark.parametrize("fam,d,tol", [(G.GAUSSIAN, 3, 1e-10), (G.PRODUCT_PEAK, 2, 1e-9),
                                       (G.C0, 2, 1e-7), (G.OSCILLATORY, 4, 1e-8),
                                       (G.CORNER_PEAK, 3, 1e-8), (G.DISCONTINUOUS, 2, 1e-4)])
def test_gk_e2e_against_oracle(oracle, gpu_ctx, fam, d, tol):
    from paper_2511_01573_gb300 import gmq
    a, u = _params(fam, d, 7)
    o = oracle.integrate(fam, a, u, tol, max_regions=1 << 16, rule=oracle.RULE_GK)
    r = gpu_ctx.integrate(fam, a, u, tol, max_regions=1 << 16, rule=gmq.RULE_GAUSS_KRONROD)
    if o.near_ties == 0:
        assert (r.status, r.iterations, r.regions_evaluated) == (o.status, o.iterations,
                                                                 o.regions_evaluated)
    assert r.function_evals == r.regions_evaluated * 15 ** d
    assert abs(r.integral - o.integral) <= 1e-12 * abs(o.integral)
    if fam != G.DISCONTINUOUS and r.status == 0:
        ex = CF.exact(fam, a, u)
        assert abs(r.integral - ex) <= 10 * tol * abs(ex)


def test_gk_batch_rejected(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    a, u = _params(G.GAUSSIAN, 3)
    import ctypes as C
    # the batched form runs the Genz-Malik rule only
    hs = [gmq._ProblemHandle(G.GAUSSIAN, a, u, None, None, 3)]
    arr = (gmq.Problem * 1)(*[x.s for x in hs])
    tols = np.array([1e-6])
    o = gmq.Options(0.0, 1e-16, 1 << 20, 0, 0, gmq.FP64, gmq.VOLUME_SHARE, 0, 0,
                    gmq.RULE_GAUSS_KRONROD)
    res = (gmq.Result * 1)()
    code = gmq.lib().gmq_integrate_batch(gpu_ctx.h, 1, arr, tols.ctypes.data_as(gmq._dp),
                                         C.byref(o), 0, res)
    assert code == gmq.ERR_INVALID
