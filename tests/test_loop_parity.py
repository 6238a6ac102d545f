"""The end-to-end comparison helper (tests/loop_parity.py) itself: it passes
on two identical runs and fails on every planted mismatch.  Mistakes are
planted in a copy of the oracle's own result, on the CPU."""
import copy

import pytest

from paper_2511_01573_gb300 import genz_inputs as G
from tests.loop_parity import assert_loop_parity, first_flagged_sweep


@pytest.fixture(scope="module")
def runs(oracle):
    a, u = G.seed_genz(1, G.C0, 4, 2.0)
    clean = oracle.integrate(G.C0, a, u, 1e-6, max_regions=1 << 20)
    a6, u6 = G.seed_genz(5, G.POLY_SUMSQ11, 5, 2.0)
    tied = oracle.integrate(G.POLY_SUMSQ11, a6 * 0, u6 * 0, 1e-5, max_regions=1 << 20)
    return clean, tied


def _gpu_like(o):
    g = copy.deepcopy(o)
    tr = [dict(t) for t in o.trace]
    return g, tr


def test_identical_runs_pass(runs):
    for o in runs:
        g, tr = _gpu_like(o)
        assert assert_loop_parity(o, g, tr) == first_flagged_sweep(o.trace)


def test_planted_mismatches_fail(runs):
    o = runs[0]
    assert first_flagged_sweep(o.trace) == len(o.trace)
    cases = []
    g, tr = _gpu_like(o)
    g.integral *= 1 + 1e-9
    cases.append((g, tr))
    g, tr = _gpu_like(o)
    g.error *= 1 + 1e-4  # 2e-11 of |I|
    cases.append((g, tr))
    g, tr = _gpu_like(o)
    tr[2]["n_split"] += 1
    cases.append((g, tr))
    g, tr = _gpu_like(o)
    tr[3]["n"] += 2
    cases.append((g, tr))
    g, tr = _gpu_like(o)
    tr[1]["I"] *= 1 + 1e-10
    cases.append((g, tr))
    g, tr = _gpu_like(o)
    g.iterations += 1
    g.regions_evaluated += 10
    tr.append(dict(tr[-1]))
    cases.append((g, tr))
    for g, tr in cases:
        with pytest.raises(AssertionError):
            assert_loop_parity(o, g, tr)


def test_flagged_run_still_checks_up_to_the_flag(runs):
    o = runs[1]
    k = first_flagged_sweep(o.trace)
    assert k < len(o.trace)  # the symmetric polynomial takes exact axis ties
    g, tr = _gpu_like(o)
    tr[k]["n"] += 2  # the flagged sweep still evaluates the same list
    with pytest.raises(AssertionError):
        assert_loop_parity(o, g, tr)
    g, tr = _gpu_like(o)
    g.integral *= 1 + 1e-9  # same decisions: the integral is still compared
    with pytest.raises(AssertionError):
        assert_loop_parity(o, g, tr)
