"""The constant tables of the library's FP64 exponential and cosine
(csrc/gm_math_tables.cuh): the committed file is what its generator writes,
and every entry agrees with the host's libm to within one ulp (the generator
rounds values computed with 60 decimal digits, libm is within an ulp), the
reduction constants split ln2/256 and pi/128 as documented."""
import math
import os
import re
import runpy

import numpy as np

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2511_01573_gb300", "csrc")


def _committed():
    with open(os.path.join(CSRC, "gm_math_tables.cuh")) as f:
        return f.read()


def _array(text, name):
    m = re.search(name + r"\[(\d+)\] = \{(.*?)\};", text, re.S)
    vals = [float(v) for v in m.group(2).replace("\n", " ").split(",") if v.strip()]
    assert len(vals) == int(m.group(1))
    return np.array(vals)


def _scalar(text, name):
    return float(re.search(r"constexpr \w+ " + name + r" = ([^;]+);", text).group(1))


def test_generator_reproduces_committed_tables(tmp_path, monkeypatch):
    monkeypatch.chdir(tmp_path)
    runpy.run_path(os.path.join(CSRC, "gen_math_tables.py"), run_name="__main__")
    with open(tmp_path / "gm_math_tables.cuh") as f:
        assert f.read() == _committed()


def test_table_entries_against_libm():
    t = _committed()
    n_exp = 1 << int(_scalar(t, "kExpTabBits"))
    n_cos = 1 << int(_scalar(t, "kCosTabBits"))
    e = _array(t, "kExp2Tab")
    c = _array(t, "kCosTab")
    s = _array(t, "kSinTab")
    assert len(e) == n_exp and len(c) == n_cos and len(s) == n_cos
    j = np.arange(n_exp)
    ref = np.exp2(j / n_exp)
    assert np.all(np.abs(e - ref) <= np.spacing(ref))
    assert e[0] == 1.0 and e[n_exp // 2] == math.sqrt(2.0)
    th = 2 * np.pi * np.arange(n_cos) / n_cos
    dth = np.spacing(th)  # the angle itself is rounded in FP64
    assert np.all(np.abs(c - np.cos(th)) <= 2.0 ** -53 + np.spacing(np.abs(c)) + dth)
    assert np.all(np.abs(s - np.sin(th)) <= 2.0 ** -53 + np.spacing(np.abs(s)) + dth)
    q = n_cos // 4  # exact zeros and ones at the quarter turns
    assert (c[0], s[0], c[q], s[q], c[2 * q], s[2 * q]) == (1.0, 0.0, 0.0, 1.0, -1.0, 0.0)
    assert np.all(c ** 2 + s ** 2 - 1.0 <= 4e-16)


def test_reduction_constants():
    t = _committed()
    n_exp = 1 << int(_scalar(t, "kExpTabBits"))
    n_cos = 1 << int(_scalar(t, "kCosTabBits"))
    l1, l2 = _scalar(t, "kExpL1"), _scalar(t, "kExpL2")
    assert abs((l1 + l2) - math.log(2.0) / n_exp) <= 1e-18
    m, _ = math.frexp(l1)
    assert (m * 2 ** 36).is_integer()          # 36 significant bits
    assert abs(l2) < 2.0 ** -35 * l1
    p1, p2 = _scalar(t, "kCosP1"), _scalar(t, "kCosP2")
    assert abs((p1 + p2) - 2 * math.pi / n_cos) <= 1e-18
    m, _ = math.frexp(p1)
    assert (m * 2 ** 33).is_integer()          # 33 significant bits
    assert _scalar(t, "kExpInvL") == n_exp / math.log(2.0)
    assert abs(_scalar(t, "kCosInvQ") - n_cos / (2 * math.pi)) <= np.spacing(n_cos / (2 * math.pi))
