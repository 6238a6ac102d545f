"""The library's FP64 exponential (Tang's table-driven method, used by the
Gaussian, C0 and discontinuous integrands), cosine (table-driven, used by
the oscillatory integrand) and reciprocal (Newton-Raphson from the hardware
approximation, used by the product-peak and corner-peak integrands) against
the host's arithmetic and CUDA's: within 2 ulp (exp), 4 units of 2^-53
absolute (cos) and 1 ulp (reciprocal) on random arguments over the whole
fast range, at the reduction boundaries and at the edges of the fallback to
the library routine."""
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
        np.log(2.0) / 512 * np.arange(-256, 257),    # reduction boundaries
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


def test_cos_accuracy(gpu_ctx):
    """Absolute error within 4 units of 2^-53 of the correctly rounded value
    (the table-driven scheme is not relatively accurate next to the zeros of
    cos, which the quadrature sums do not need), 2 ulp where |cos x| >= 1/2."""
    rng = np.random.default_rng(7)
    x = np.concatenate([
        rng.uniform(-100.0, 100.0, 1 << 20),
        rng.uniform(0.0, 15.0, 1 << 18),             # the oscillatory family's range
        rng.uniform(-99999.0, 99999.0, 1 << 16),
        np.pi / 256 * np.arange(-800, 801) + 1e-12,  # reduction boundaries
        np.array([0.0, -0.0, 1e-300, np.pi / 2, np.pi, 1e5, -1e5, 1e6, np.inf, np.nan]),
    ])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    y = gpu_ctx.math_cos(xd).cpu().numpy()
    ref_cuda = torch.cos(xd).cpu().numpy()
    ref_host = np.cos(x)
    fast = np.abs(x) < 1e5
    assert np.max(np.abs(y[fast] - ref_host[fast])) <= 4 * 2.0 ** -53
    assert np.max(np.abs(y[fast] - ref_cuda[fast])) <= 4 * 2.0 ** -53
    big = fast & (np.abs(ref_host) >= 0.5)
    assert np.max(_ulps(y[big], ref_host[big])) <= 2.0
    slow = ~fast
    assert np.array_equal(y[slow], ref_cuda[slow], equal_nan=True)
