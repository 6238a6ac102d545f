"""Mixed form (FP32 integrand, TwoSum-compensated FP32 class sums, FP64
differences, axis choice and global sums) against the FP64 oracle.

The mixed form is not expected to match the oracle to 1e-12: node values
carry FP32 rounding (about 6e-8 relative each), so the per-region rule value
is compared with a 5e-6 bound relative to the magnitude of its terms (the
oscillatory family's FP32 argument, up to 2 pi + sum a_j, carries an absolute
rounding of about 1e-6) and
the end-to-end integral with max(tol, 2e-6) relative.  The errors measured
here are the ones reported for the mixed form.
"""
import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G
from tests import closed_forms as CF

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MIXED = 1


def _soa(x):
    return torch.tensor(np.ascontiguousarray(x.T), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("fam", [G.OSCILLATORY, G.PRODUCT_PEAK, G.CORNER_PEAK, G.GAUSSIAN, G.C0])
@pytest.mark.parametrize("d,lanes", [(3, 1), (8, 1), (8, 4), (8, 32), (12, 1)])
def test_mixed_rule_per_region(oracle, gpu_ctx, fam, d, lanes):
    a, u = G.seed_genz(3, fam, d, 5.0 * d if fam == G.PRODUCT_PEAK else G.GENZ_TARGET_SUM[fam])
    n = {3: 1000, 8: 120, 12: 10}[d]
    c, h = G.random_boxes(9 + d, n, d)
    o = oracle.rule_regions(fam, a, u, c, h)
    i7, err, vf, ax = gpu_ctx.eval_rule(fam, a, u, _soa(c), _soa(h), precision=MIXED, lanes=lanes)
    i7 = i7.cpu().numpy()
    rel = np.abs(i7 - o["i7"]) / o["i7abs"]
    assert rel.max() <= 5e-6, rel.max()
    assert np.array_equal(vf.cpu().numpy(), o["vol"])


@pytest.mark.parametrize("fam", G.GENZ_D8_FAMILIES)
@pytest.mark.parametrize("tol", [1e-4, 1e-6])
def test_mixed_e2e_d8_against_closed_form(gpu_ctx, fam, tol):
    a, u = G.seed_genz(1, fam, 8, G.GENZ_TARGET_SUM[fam])
    ex = CF.exact(fam, a, u)
    r64 = gpu_ctx.integrate(fam, a, u, tol, max_regions=1 << 24)
    rmx = gpu_ctx.integrate(fam, a, u, tol, max_regions=1 << 24, precision=MIXED)
    assert rmx.status in (0, 1, 3)
    err_mx = abs(rmx.integral - ex) / abs(ex)
    err_64 = abs(r64.integral - ex) / abs(ex)
    allowed = max(tol, 2e-6) * (10 if fam == G.GAUSSIAN else 1)
    assert err_mx <= allowed, (err_mx, err_64)
    print(f"{G.FAMILY_NAMES[fam]} tol={tol:g}: mixed rel err {err_mx:.2e} "
          f"(fp64 {err_64:.2e}), regions {rmx.regions_evaluated} vs {r64.regions_evaluated}")


def test_mixed_e2e_d3_product_peak(gpu_ctx, oracle):
    p = G.product_peak_d3()
    o = oracle.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=100000)
    r = gpu_ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=100000, precision=MIXED)
    assert r.status == 0
    assert abs(r.integral - o.integral) <= 2e-6 * abs(o.integral)
