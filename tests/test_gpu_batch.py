"""Batched form (gmq_integrate_batch) on the GPU.

Every problem of a batch must get exactly the result gmq_integrate gives it
alone (the same per-region arithmetic, sums, decisions and child order,
whatever lanes per region either side uses): integral, error, region count,
sweeps and status are compared for equality, in the CUDA-graph mode and in
the host-driven mode, with the autotuned per-sweep mapping and with each
mapping forced.
The single-problem path is itself checked against the CPU oracle in
test_gpu_parity.py; here a sample of batch results is also checked against
the oracle directly.
"""
import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mixed_batch(n=48, seed=7):
    g = G.SplitMix64(seed)
    out = []
    for i in range(n):
        d = 2 + int(g.next_u64() % 7)
        fam = G.GENZ_D8_FAMILIES[g.next_u64() % 4]
        tol = 10.0 ** (-3.0 - 4.0 * g.next_double())
        a, u = G.seed_genz(seed * 1000 + i, fam, d, G.GENZ_TARGET_SUM[fam])
        out.append(G.Problem(fam, d, a, u, tol))
    return out


def _single(gpu_ctx, p, cap):
    return gpu_ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=cap, lanes=1)


@pytest.mark.parametrize("host_loop", [False, True])
def test_batch_equals_single_runs(gpu_ctx, host_loop):
    probs = _mixed_batch()
    cap = 1 << 22
    res = gpu_ctx.integrate_batch(probs, max_regions=cap, host_loop=host_loop)
    info = gpu_ctx.last_batch_info()
    assert info["used_graph"] == (not host_loop)
    assert info["rule_block"] == 128
    assert sum(info["lane_sweeps"]) == info["sweeps"]
    for p, r in zip(probs, res):
        s = _single(gpu_ctx, p, cap)
        assert (r.status, r.iterations, r.regions_evaluated) == (s.status, s.iterations,
                                                                 s.regions_evaluated), p.label
        assert r.integral == s.integral and r.error == s.error
    assert info["sweeps"] >= max(r.iterations for r in res)


@pytest.mark.parametrize("lanes", [1, 4, 32, 128])
def test_batch_forced_lane_mappings(gpu_ctx, lanes):
    probs = _mixed_batch(n=24, seed=13)
    cap = 1 << 20
    res = gpu_ctx.integrate_batch(probs, max_regions=cap, lanes=lanes)
    info = gpu_ctx.last_batch_info()
    assert info["forced_lanes"] == lanes and not info["autotuned"]
    assert info["lane_sweeps"][{1: 0, 4: 1, 32: 2, 128: 3}[lanes]] == info["sweeps"]
    for p, r in zip(probs, res):
        s = gpu_ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=cap)
        assert (r.status, r.iterations, r.regions_evaluated) == (s.status, s.iterations,
                                                                 s.regions_evaluated), p.label
        assert r.integral == s.integral and r.error == s.error


def _mixed_precision_batch():
    probs = _mixed_batch(n=32, seed=17)
    extra = [(G.PRODUCT_PEAK, 1, 1e-6), (G.GAUSSIAN, 12, 1e-3), (G.C0, 13, 1e-2),
             (G.DISCONTINUOUS, 3, 1e-3), (G.POLY_SUMSQ11, 2, 1e-5), (G.OSCILLATORY, 10, 1e-4)]
    for i, (fam, d, tol) in enumerate(extra):
        a, u = G.seed_genz(900 + i, fam, d, G.GENZ_TARGET_SUM.get(fam, 2.0))
        if fam == G.PRODUCT_PEAK:
            a, u = G.seed_genz(900 + i, fam, d, 5.0)
        if fam == G.DISCONTINUOUS:
            u = 0.3 + 0.6 * u
        probs.append(G.Problem(fam, d, a, u, tol))
    return probs


@pytest.mark.parametrize("host_loop", [False, True])
def test_batch_mixed_equals_single_mixed(gpu_ctx, host_loop):
    """Mixed form: one lane per region, the single path's per-region code
    (register walk for 3 <= d <= 12, generic otherwise), so every problem
    gets the bits of gmq_integrate's mixed form with lanes = 1."""
    from paper_2511_01573_gb300 import gmq
    probs = _mixed_precision_batch()
    cap = 1 << 20
    res = gpu_ctx.integrate_batch(probs, max_regions=cap, precision=gmq.MIXED,
                                  host_loop=host_loop)
    info = gpu_ctx.last_batch_info()
    assert info["forced_lanes"] == 1 and info["lane_sweeps"][0] == info["sweeps"]
    for p, r in zip(probs, res):
        s = gpu_ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=cap, lanes=1,
                              precision=gmq.MIXED)
        assert (r.status, r.iterations, r.regions_evaluated) == (s.status, s.iterations,
                                                                 s.regions_evaluated), p.label
        assert r.integral == s.integral and r.error == s.error
    with pytest.raises(gmq.GmqError):
        gpu_ctx.integrate_batch(probs[:4], precision=gmq.MIXED, lanes=4)


def test_batch_against_oracle_sample(oracle, gpu_ctx):
    probs = _mixed_batch(n=12, seed=11)
    res = gpu_ctx.integrate_batch(probs, max_regions=1 << 20)
    for p, r in zip(probs, res):
        o = oracle.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=1 << 20)
        if o.near_ties == 0:
            assert (r.status, r.iterations, r.regions_evaluated) == (o.status, o.iterations,
                                                                     o.regions_evaluated)
        assert abs(r.integral - o.integral) <= 1e-12 * abs(o.integral)


def test_batch_many_integrals_workload_sample(gpu_ctx):
    """The first 128 of the 4096-integral workload (d ~ U{2..10}, four
    families, tolerance log-uniform in [1e-9, 1e-4]); every result equals
    its single run.  The work counters add up: every sweep's list is
    evaluated or carried over, and the evaluated regions are the results'
    region counts plus the work evictions dropped."""
    probs = G.batched_problems(count=128)
    cap = 1 << 20
    # a pool far smaller than the problems' combined peak: problems wait,
    # pause and are evicted and restarted, none of which may change a result
    res = gpu_ctx.integrate_batch(probs, max_regions=cap, pool_regions=1 << 22)
    info = gpu_ctx.last_batch_info()
    assert info["pauses"] + info["evictions"] > 0
    assert info["list_regions"] == info["rule_regions"] + info["carried_regions"]
    assert (info["carried_regions"] > 0) == (info["pauses"] > 0)
    counted = sum(r.regions_evaluated for r in res)
    assert counted <= info["rule_regions"]
    if info["evictions"] == 0:
        assert counted == info["rule_regions"]
    for p, r in list(zip(probs, res))[::8]:
        s = _single(gpu_ctx, p, cap)
        assert (r.status, r.regions_evaluated, r.integral) == (s.status, s.regions_evaluated,
                                                               s.integral)


def test_batch_autotune_cached_and_limits(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    probs = _mixed_batch(n=8, seed=3)
    first = gpu_ctx.integrate_batch(probs)
    info = gpu_ctx.last_batch_info()
    if info["autotuned"]:
        tune = info["tune"]
        assert 1 <= len(tune) <= 5 and all(len(t["ms"]) == 4 for t in tune)
        assert all(t["ms"][m] > 0 for t in tune for m in range(4))
        assert [t["n"] for t in tune] == sorted(t["n"] for t in tune)
    assert 0 <= info["lanes_t32"] <= info["lanes_t4"] <= info["lanes_t1"]
    again = gpu_ctx.integrate_batch(probs)
    assert not gpu_ctx.last_batch_info()["autotuned"]  # cached per largest dimension
    assert [(r.integral, r.regions_evaluated) for r in again] == [
        (r.integral, r.regions_evaluated) for r in first]
    # sweep limit: every problem stops by the third sweep
    res = gpu_ctx.integrate_batch(probs, max_iters=3)
    assert all(r.iterations <= 3 for r in res)
    assert all(r.status in (0, 2) for r in res)
    # pool overflow: the running problems stop with CAP_REACHED
    hard = [G.Problem(G.C0, 6, *G.seed_genz(1, G.C0, 6, 2.0), 1e-9)] * 4
    res = gpu_ctx.integrate_batch(hard, max_regions=1 << 20, pool_regions=1 << 15)
    assert all(r.status == gmq.CAP_REACHED for r in res)
    # invalid arguments
    with pytest.raises(gmq.GmqError):
        # an initial partition larger than half the pool could never start
        gpu_ctx.integrate_batch(probs, pool_regions=64)
    with pytest.raises(gmq.GmqError):
        gpu_ctx.integrate_batch(probs, lanes=8)
    with pytest.raises(gmq.GmqError):
        # the device loop's bound 4 x max_iters must fit an int
        gpu_ctx.integrate_batch(probs, max_iters=(1 << 28) + 1)
    assert len(again) == len(probs)
