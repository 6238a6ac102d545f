"""Seeded synthetic inputs for the Genz test families.

This module only draws numbers: it holds none of the quadrature method's
arithmetic, so both the CUDA path and the CPU oracle may take their inputs
from it.  The library exports the same generator as ``gmq_seed_genz``; the
two are written independently and a test checks that they agree bit for bit.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), one stream per (seed, family, dim) with
initial state ``(seed << 16) ^ (family << 8) ^ dim``.  Each draw advances the
state by the golden-ratio increment and mixes it; a double in [0, 1) is the
top 53 bits times 2^-53.  The stream gives a_1..a_d, then u_1..u_d; the a_j
are then rescaled so that sum_j a_j equals the requested target
(a_j * (target / sum_k a_k)), which is how Genz sets a family's difficulty.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15

# family codes (identical numbering to the C ABI)
OSCILLATORY = 0
PRODUCT_PEAK = 1
CORNER_PEAK = 2
GAUSSIAN = 3
C0 = 4
DISCONTINUOUS = 5
POLY_SUMSQ11 = 6

FAMILY_NAMES = {
    OSCILLATORY: "oscillatory",
    PRODUCT_PEAK: "product_peak",
    CORNER_PEAK: "corner_peak",
    GAUSSIAN: "gaussian",
    C0: "c0",
    DISCONTINUOUS: "discontinuous",
    POLY_SUMSQ11: "poly_sumsq11",
}

# difficulty (sum of a_j) of the four seeded families of the d=8 workload,
# in the order oscillatory, Gaussian, corner peak, C0
GENZ_TARGET_SUM = {OSCILLATORY: 6.0, GAUSSIAN: 3.5, CORNER_PEAK: 1.85, C0: 2.0}


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


class SplitMix64:
    """SplitMix64 stream; ``next_u64`` then ``next_double`` in [0, 1)."""

    def __init__(self, state: int):
        self.state = state & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GAMMA) & _MASK
        return _mix(self.state)

    def next_double(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


def stream_state(seed: int, family: int, dim: int) -> int:
    return ((seed << 16) ^ (family << 8) ^ dim) & _MASK


def seed_genz(seed: int, family: int, dim: int, target_sum: float):
    """a_j ~ U(0,1) rescaled to sum target_sum, u_j ~ U(0,1)."""
    g = SplitMix64(stream_state(seed, family, dim))
    a = [g.next_double() for _ in range(dim)]
    u = [g.next_double() for _ in range(dim)]
    tot = 0.0
    for v in a:
        tot = tot + v
    scale = target_sum / tot
    a = [v * scale for v in a]
    return np.array(a, dtype=np.float64), np.array(u, dtype=np.float64)


def seed_uniform(seed: int, family: int, dim: int, a_lo: float, a_hi: float):
    """a_j ~ U(a_lo, a_hi), u_j ~ U(0,1) on the same stream layout."""
    g = SplitMix64(stream_state(seed, family, dim))
    a = [a_lo + (a_hi - a_lo) * g.next_double() for _ in range(dim)]
    u = [g.next_double() for _ in range(dim)]
    return np.array(a, dtype=np.float64), np.array(u, dtype=np.float64)


@dataclass
class Problem:
    family: int
    dim: int
    a: np.ndarray
    u: np.ndarray
    rel_tol: float
    lo: np.ndarray = field(default=None)
    hi: np.ndarray = field(default=None)
    label: str = ""

    def __post_init__(self):
        if self.lo is None:
            self.lo = np.zeros(self.dim)
        if self.hi is None:
            self.hi = np.ones(self.dim)


def product_peak_d3() -> Problem:
    """Product peak on [0,1]^3, a_j = 5, u_j = 1/2, rel tol 1e-6 (cap 1e5)."""
    return Problem(PRODUCT_PEAK, 3, np.full(3, 5.0), np.full(3, 0.5), 1e-6,
                   label="product_peak_d3_a5")


GENZ_D8_FAMILIES = (OSCILLATORY, GAUSSIAN, CORNER_PEAK, C0)
GENZ_D8_TOLS = (1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8)


def genz_d8_problems(seeds=range(1, 11), tols=GENZ_D8_TOLS, families=GENZ_D8_FAMILIES):
    """Four Genz families on [0,1]^8, seeds 1..10, rel tol 1e-3..1e-8."""
    out = []
    for tol in tols:
        for fam in families:
            for s in seeds:
                a, u = seed_genz(s, fam, 8, GENZ_TARGET_SUM[fam])
                out.append(Problem(fam, 8, a, u, tol,
                                   label=f"{FAMILY_NAMES[fam]}_d8_s{s}_tol{tol:g}"))
    return out


def genz_d12_problems(seeds=range(1, 11), tols=(1e-4, 1e-5, 1e-6, 1e-7)):
    """Corner peak and Gaussian on [0,1]^12 (4409 nodes per region)."""
    out = []
    for tol in tols:
        for fam in (CORNER_PEAK, GAUSSIAN):
            for s in seeds:
                a, u = seed_genz(s, fam, 12, GENZ_TARGET_SUM[fam])
                out.append(Problem(fam, 12, a, u, tol,
                                   label=f"{FAMILY_NAMES[fam]}_d12_s{s}_tol{tol:g}"))
    return out


def paper_integrand(index: int, dim: int) -> Problem:
    """The paper's test functions f1..f7 on [0,1]^d as family instances."""
    j = np.arange(1, dim + 1, dtype=np.float64)
    if index == 1:
        return Problem(OSCILLATORY, dim, j.copy(), np.zeros(dim), 1e-6, label="f1")
    if index == 2:
        return Problem(PRODUCT_PEAK, dim, np.full(dim, 50.0), np.full(dim, 0.5), 1e-6, label="f2")
    if index == 3:
        return Problem(CORNER_PEAK, dim, j.copy(), np.zeros(dim), 1e-6, label="f3")
    if index == 4:
        return Problem(GAUSSIAN, dim, np.full(dim, 25.0), np.full(dim, 0.5), 1e-6, label="f4")
    if index == 5:
        return Problem(C0, dim, np.full(dim, 10.0), np.full(dim, 0.5), 1e-6, label="f5")
    if index == 6:
        return Problem(DISCONTINUOUS, dim, j + 4.0, (3.0 + j) / 10.0, 1e-6, label="f6")
    if index == 7:
        return Problem(POLY_SUMSQ11, dim, np.zeros(dim), np.zeros(dim), 1e-6, label="f7")
    raise ValueError(index)


def batched_problems(count=4096, master_seed=2511):
    """Many independent integrals: d ~ U{2..10}, family ~ U of the four Genz
    families, rel tol log-uniform in [1e-9, 1e-4], all from one master seed."""
    g = SplitMix64(master_seed)
    out = []
    for i in range(count):
        dim = 2 + (g.next_u64() % 9)
        fam = GENZ_D8_FAMILIES[g.next_u64() % 4]
        tol = 10.0 ** (-4.0 - 5.0 * g.next_double())
        a, u = seed_genz(master_seed * 8192 + i, fam, int(dim), GENZ_TARGET_SUM[fam])
        out.append(Problem(fam, int(dim), a, u, tol, label=f"batch{i}"))
    return out


def gaussian_grad_sets(count=1024, dim=6, master_seed=1):
    """Gaussian family parameter sets with a_j ~ U(0.5, 3), u_j ~ U(0, 1)."""
    return [seed_uniform(master_seed * 65536 + i, GAUSSIAN, dim, 0.5, 3.0) for i in range(count)]


def random_dyadic_boxes(seed: int, n: int, dim: int):
    """n random sub-boxes of [0,1]^dim shaped like the regions a refinement
    leaves (AoS, n x d): per axis the half-width is 2^-j, j uniform in
    1..12, and the centre is uniform over the positions that keep the box in
    [0,1].  Vectorised (numpy's PCG64 seeded with `seed`), for lists of
    millions of regions."""
    rng = np.random.default_rng(seed)
    j = rng.integers(1, 13, size=(n, dim)).astype(np.int32)
    h = np.ldexp(1.0, -j)
    c = h + (1.0 - 2.0 * h) * rng.random((n, dim))
    return c, h


def random_boxes(seed: int, n: int, dim: int, lo=0.0, hi=1.0):
    """n random sub-boxes of [lo,hi]^dim: centres and half-widths (AoS, n x d)."""
    g = SplitMix64(stream_state(seed, 255, dim))
    c = np.empty((n, dim))
    h = np.empty((n, dim))
    for r in range(n):
        for k in range(dim):
            x0 = lo + (hi - lo) * g.next_double()
            x1 = lo + (hi - lo) * g.next_double()
            a, b = min(x0, x1), max(x0, x1)
            if b - a < 1e-3:
                b = a + 1e-3
            c[r, k] = 0.5 * (a + b)
            h[r, k] = 0.5 * (b - a)
    return c, h

