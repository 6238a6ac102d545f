"""The library's FP64 exponential (Tang's table-driven method, used by the
Gaussian, C0 and discontinuous integrands) and reciprocal (Newton-Raphson
from the hardware approximation, used by the product-peak and corner-peak
integrands) against the host's arithmetic and CUDA's: within 2 ulp (exp)
and 1 ulp (reciprocal) on random arguments over the whole fast range and at
the edges of the fallback to the library routine."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ulps(a, b):
    """|a - b| in units of the last place of b."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_exp_accuracy(gpu_ctx):
    rng = np.random.default_rng(2511)
    x = np.concatenate([
        rng.uniform(-707.0, 707.0, 1 << 20),
        rng.uniform(-1.0, 1.0, 1 << 18),
        rng.uniform(-20.0, 0.0, 1 << 18),           # the integrands' usual range
        np.array([0.0, -0.0, 1e-300, -1e-300, 5e-324, 1.0, -1.0, 706.99, -706.99,
                  707.0, -707.0, 708.5, -708.5, 709.7, -745.0, -746.0, 710.0]),
        np.log(2.0) / 128 * np.arange(-64, 65),      # reduction boundaries
    ])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = gpu_ctx.math_exp(xd).cpu().numpy()
    ref_host = np.exp(x)
    ref_cuda = torch.exp(xd).cpu().numpy()
    finite = np.isfinite(ref_host) & (ref_host > np.finfo(np.float64).tiny)
    assert np.max(_ulps(y[finite], ref_host[finite])) <= 2.0
    assert np.max(_ulps(y[finite], ref_cuda[finite])) <= 2.0
    # outside the fast range the library exp itself is used
    edge = ~finite
    assert np.array_equal(y[edge], ref_cuda[edge])
    assert np.all(y[x == 0.0] == 1.0)
    nan = gpu_ctx.math_exp(torch.tensor([np.nan], dtype=torch.float64, device="cuda"))
    assert torch.isnan(nan).all()


def test_rcp_accuracy(gpu_ctx):
    rng = np.random.default_rng(1573)
    mag = np.exp2(rng.uniform(-119.9, 119.9, 1 << 20))
    x = np.concatenate([
        mag * np.where(rng.random(mag.size) < 0.5, -1.0, 1.0),
        rng.uniform(1.0, 2.0, 1 << 18),
        np.array([1.0, -1.0, 2.0, 0.5, 3.0, 2.0 ** -120, 2.0 ** 120, 2.0 ** -121, 2.0 ** 121,
                  2.0 ** -1070, 1e300, -1e-300, 0.0, -0.0, np.inf, -np.inf]),
    ])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = gpu_ctx.math_rcp(xd).cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        ref = 1.0 / x  # IEEE division: correctly rounded
    fast = np.abs(x) >= 2.0 ** -120
    fast &= np.abs(x) <= 2.0 ** 120
    assert np.max(_ulps(y[fast], ref[fast])) <= 1.0
    slow = ~fast
    assert np.array_equal(y[slow], ref[slow])
