"""Closed-form integrals of the built-in families over [0,1]^d.

Independent of both the oracle and the CUDA path: each is the textbook
antiderivative of the family (paper Sec. 4 integrands; Genz families).
With mpmath available the values are computed at 50 digits (the corner-peak
inclusion-exclusion sum cancels badly in FP64); otherwise in double.
"""
import math
from fractions import Fraction
from itertools import combinations

try:
    import mpmath as mp
    mp.mp.dps = 50
except ImportError:  # mpmath is optional; without it the forms run in FP64
    mp = None

OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS, POLY_SUMSQ11 = range(7)


def _f(x):
    return mp.mpf(float(x)) if mp else float(x)


def oscillatory(a, u):
    # Re[ e^{i 2 pi u_1} prod_j (e^{i a_j} - 1) / (i a_j) ]
    if mp:
        z = mp.expj(2 * mp.pi * _f(u[0]))
        for aj in a:
            aj = _f(aj)
            z *= (mp.expj(aj) - 1) / (1j * aj)
        return float(mp.re(z))
    z = complex(math.cos(2 * math.pi * u[0]), math.sin(2 * math.pi * u[0]))
    for aj in a:
        z *= (complex(math.cos(aj), math.sin(aj)) - 1) / (1j * aj)
    return z.real


def product_peak(a, u):
    out = _f(1)
    for aj, uj in zip(a, u):
        aj, uj = _f(aj), _f(uj)
        at = mp.atan if mp else math.atan
        out *= aj * (at(aj * (1 - uj)) + at(aj * uj))
    return float(out)


def corner_peak(a):
    d = len(a)
    if mp:
        aa = [_f(v) for v in a]
        tot = mp.mpf(0)
        for k in range(d + 1):
            for S in combinations(range(d), k):
                tot += (-1) ** k / (1 + sum((aa[j] for j in S), mp.mpf(0)))
        den = mp.factorial(d)
        for v in aa:
            den *= v
        return float(tot / den)
    tot = 0.0
    for k in range(d + 1):
        for S in combinations(range(d), k):
            tot += (-1) ** k / (1 + sum(a[j] for j in S))
    return tot / (math.factorial(d) * math.prod(a))


def gaussian(a, u):
    out = _f(1)
    for aj, uj in zip(a, u):
        aj, uj = _f(aj), _f(uj)
        if mp:
            out *= mp.sqrt(mp.pi) / (2 * aj) * (mp.erf(aj * (1 - uj)) + mp.erf(aj * uj))
        else:
            out *= math.sqrt(math.pi) / (2 * aj) * (math.erf(aj * (1 - uj)) + math.erf(aj * uj))
    return float(out)


def c0(a, u):
    out = _f(1)
    ex = mp.exp if mp else math.exp
    for aj, uj in zip(a, u):
        aj, uj = _f(aj), _f(uj)
        out *= (2 - ex(-aj * uj) - ex(-aj * (1 - uj))) / aj
    return float(out)


def discontinuous(a, u):
    out = _f(1)
    ex = mp.exp if mp else math.exp
    for aj, uj in zip(a, u):
        aj = _f(aj)
        t = _f(min(1.0, max(0.0, float(uj))))
        out *= (ex(aj * t) - 1) / aj
    return float(out)


def poly_sumsq11(d):
    """int_[0,1]^d (sum x_j^2)^11 = sum over k_1+..+k_d = 11 of
    11!/prod k_i! * prod 1/(2 k_i + 1), exact in rationals."""
    def rec(j, left):
        if j == d - 1:
            return Fraction(1, math.factorial(left) * (2 * left + 1))
        tot = Fraction(0)
        for k in range(left + 1):
            tot += Fraction(1, math.factorial(k) * (2 * k + 1)) * rec(j + 1, left - k)
        return tot
    return float(math.factorial(11) * rec(0, 11))


def exact(family, a, u):
    d = len(a)
    if family == OSCILLATORY:
        return oscillatory(a, u)
    if family == PRODUCT_PEAK:
        return product_peak(a, u)
    if family == CORNER_PEAK:
        return corner_peak(a)
    if family == GAUSSIAN:
        return gaussian(a, u)
    if family == C0:
        return c0(a, u)
    if family == DISCONTINUOUS:
        return discontinuous(a, u)
    if family == POLY_SUMSQ11:
        return poly_sumsq11(d)
    raise ValueError(family)
