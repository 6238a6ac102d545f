"""Writes gm_math_tables.cuh: the constants of the library's FP64 exponential
and cosine (gmq_families.cuh, gm_exp and gm_cos), computed in decimal
arithmetic with 60 significant digits.

Method: Tang's table-driven exponential (P. T. P. Tang, ACM TOMS 15(2),
1989).  x = (2048 m + j) ln2/2048 + r, |r| <= ln2/4096, exp(x) = 2^m
2^(j/2048) exp(r).  The table holds 2^(j/2048), j = 0..2047, rounded to
nearest; ln2/2048 is split into L1 (36 significant bits) and L2 = ln2/2048
- L1 rounded; exp(r) - 1 is the Taylor polynomial of degree 3 (its
truncation error r^4/24 is below 3.5e-17).

Cosine, by the same table-driven scheme (J.-M. Muller, Elementary Functions,
ch. 6): x = n pi/128 + r, |r| <= pi/256, cos(x) = C_j cos(r) - S_j sin(r)
with j = n mod 256, C_j = cos(j pi/128), S_j = sin(j pi/128); pi/128 is
split into P1 (33 significant bits) and P2 = pi/128 - P1 rounded.  With
fused multiply-adds the first step x - n P1 is exact (the result is a
multiple of the coarser of ulp(x) and P1's last bit, and no larger than
|x|), and the second leaves an error n |pi/128 - P1 - P2| below 2^-70 for
|n| < 2^22, so two parts suffice.

Run from this directory: python gen_math_tables.py
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


def dec_pi():
    # Machin: pi = 16 atan(1/5) - 4 atan(1/239)
    def atan_inv(q):
        s, t, k = Decimal(0), Decimal(1) / q, 0
        while abs(t) > Decimal(10) ** -59:
            s += t / (2 * k + 1) * (-1) ** k
            t /= q * q
            k += 1
        return s
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def dec_cos_sin(x):
    c, s, t, k = Decimal(0), Decimal(0), Decimal(1), 0
    while abs(t) > Decimal(10) ** -58 or k < 4:
        if k % 4 == 0:
            c += t
        elif k % 4 == 1:
            s += t
        elif k % 4 == 2:
            c -= t
        else:
            s -= t
        k += 1
        t = t * x / k
    return c, s


def split_bits(d: Decimal, bits: int) -> float:
    m, e = math.frexp(float(d))
    scale = Decimal(2) ** (bits - e)
    return float((d * scale).to_integral_value() / scale)


def to_double(d: Decimal) -> float:
    """Round a Decimal to the nearest double (ties to even)."""
    f = float(d)  # correctly rounded: Python converts via the exact decimal string
    return f


def split36(d: Decimal) -> float:
    """d rounded to 36 significant bits."""
    m, e = math.frexp(float(d))
    scale = Decimal(2) ** (36 - e)
    return float((d * scale).to_integral_value() / scale)


NEXP = 2048  # table entries of the exponential (2^(j/NEXP))
NCOS = 256  # table entries of the cosine (cos, sin of 2 pi j/NCOS)


def main():
    ln2 = dec_ln2()
    c = ln2 / NEXP
    l1 = split36(c)
    l2 = to_double(c - Decimal(l1))
    inv = to_double(NEXP / ln2)
    tab = [to_double(dec_exp(ln2 * j / NEXP)) for j in range(NEXP)]
    pi = dec_pi()
    q = 2 * pi / NCOS
    p1 = split_bits(q, 33)
    p2 = to_double(q - Decimal(p1))
    invq = to_double(NCOS / (2 * pi))
    # cos and sin of 2 pi j/NCOS; the exact zeros (j = 0, NCOS/4, NCOS/2,
    # 3 NCOS/4) come out of the series as residues below 1e-40 and are set to 0
    cs = [tuple(Decimal(0) if abs(v) < Decimal(10) ** -40 else v
                for v in dec_cos_sin(2 * pi * j / NCOS))
          for j in range(NCOS)]
    lines = [
        "// gm_math_tables.cuh -- generated by gen_math_tables.py (decimal arithmetic, 60",
        "// digits); constants of gm_exp and gm_cos (gmq_families.cuh).",
        "#pragma once",
        "",
        "namespace gmq {",
        "",
        f"constexpr int kExpTabBits = {NEXP.bit_length() - 1};  // {NEXP} entries",
        f"constexpr double kExpInvL = {inv!r};  // {NEXP} / ln 2",
        f"constexpr double kExpL1 = {l1!r};  // ln2/{NEXP}, 36 significant bits",
        f"constexpr double kExpL2 = {l2!r};  // ln2/{NEXP} - kExpL1",
        "",
        f"// 2^(j/{NEXP}), j = 0..{NEXP - 1}, rounded to nearest",
        f"static __device__ const double kExp2Tab[{NEXP}] = {{",
    ]
    for i in range(0, NEXP, 2):
        lines.append(f"    {tab[i]!r}, {tab[i + 1]!r},")
    lines += ["};", "",
              f"constexpr int kCosTabBits = {NCOS.bit_length() - 1};  // {NCOS} entries",
              f"constexpr double kCosInvQ = {invq!r};  // {NCOS // 2} / pi",
              f"constexpr double kCosP1 = {p1!r};  // pi/{NCOS // 2}, 33 significant bits",
              f"constexpr double kCosP2 = {p2!r};  // pi/{NCOS // 2} - P1",
              "",
              f"// cos(j pi/{NCOS // 2}) and sin(j pi/{NCOS // 2}), j = 0..{NCOS - 1}, rounded to nearest",
              f"static __device__ const double kCosTab[{NCOS}] = {{"]
    for i in range(0, NCOS, 2):
        lines.append(f"    {to_double(cs[i][0])!r}, {to_double(cs[i + 1][0])!r},")
    lines += ["};", f"static __device__ const double kSinTab[{NCOS}] = {{"]
    for i in range(0, NCOS, 2):
        lines.append(f"    {to_double(cs[i][1])!r}, {to_double(cs[i + 1][1])!r},")
    lines += ["};", "", "}  // namespace gmq", ""]
    with open("gm_math_tables.cuh", "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
