"""Writes gm_exp_table.cuh: the constants of the library's FP64 exponential
(gmq_families.cuh, gm_exp), computed in exact decimal arithmetic.

Method: Tang's table-driven exponential (P. T. P. Tang, ACM TOMS 15(2),
1989).  x = (64 m + j) ln2/64 + r, |r| <= ln2/128, exp(x) = 2^m 2^(j/64)
exp(r).  The table holds 2^(j/64), j = 0..63, rounded to nearest; ln2/64 is
split into L1 (36 significant bits, so n L1 is exact for |n| < 2^17) and
L2 = ln2/64 - L1 rounded; exp(r) - 1 is the Taylor polynomial of degree 5
(its truncation error r^6/720 is below 3.6e-17 relative).

Run from this directory: python gen_exp_table.py
"""
from decimal import Decimal, getcontext
import math

getcontext().prec = 60


def dec_ln2():
    # ln 2 = sum_{k>=1} 1 / (k 2^k)
    s, t = Decimal(0), Decimal(1)
    for k in range(1, 400):
        t /= 2
        s += t / k
    return s


def dec_exp(x):
    s, t, k = Decimal(1), Decimal(1), 0
    while True:
        k += 1
        t = t * x / k
        if abs(t) < Decimal(10) ** -58:
            return s + t
        s += t


def to_double(d: Decimal) -> float:
    """Round a Decimal to the nearest double (ties to even)."""
    f = float(d)  # correctly rounded: Python converts via the exact decimal string
    return f


def split36(d: Decimal) -> float:
    """d rounded to 36 significant bits."""
    m, e = math.frexp(float(d))
    scale = Decimal(2) ** (36 - e)
    return float((d * scale).to_integral_value() / scale)


def main():
    ln2 = dec_ln2()
    c = ln2 / 64
    l1 = split36(c)
    l2 = to_double(c - Decimal(l1))
    inv = to_double(64 / ln2)
    tab = [to_double(dec_exp(ln2 * j / 64)) for j in range(64)]
    lines = [
        "// gm_exp_table.cuh -- generated by gen_exp_table.py (exact decimal arithmetic);",
        "// constants of gm_exp (gmq_families.cuh): Tang's table-driven exponential.",
        "#pragma once",
        "",
        "namespace gmq {",
        "",
        f"constexpr double kExpInvL = {inv!r};  // 64 / ln 2",
        f"constexpr double kExpL1 = {l1!r};  // ln2/64, 36 significant bits",
        f"constexpr double kExpL2 = {l2!r};  // ln2/64 - kExpL1",
        "",
        "// 2^(j/64), j = 0..63, rounded to nearest",
        "static __device__ const double kExp2Tab[64] = {",
    ]
    for i in range(0, 64, 2):
        lines.append(f"    {tab[i]!r}, {tab[i + 1]!r},")
    lines += ["};", "", "}  // namespace gmq", ""]
    with open("gm_exp_table.cuh", "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
