"""The C-ABI library loads and exports every symbol that include/gmq.h
declares; host-only calls (no GPU needed) behave as documented."""
import os
import re

import numpy as np
import pytest

from paper_2511_01573_gb300 import genz_inputs as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gmq.h")).read()
    return sorted(set(re.findall(r"^\s*(?:gmq_status|const char \*)\s*(gmq_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_2511_01573_gb300 import build as B
    B.build()
    from paper_2511_01573_gb300 import gmq
    return gmq


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("gmq_create", "gmq_destroy", "gmq_set_stream", "gmq_set_pool", "gmq_integrate",
              "gmq_seed_genz", "gmq_status_string", "gmq_eval_rule", "gmq_classify_split"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    L = built.lib()
    for n in _declared():
        assert hasattr(L, n), n
    assert set(_declared()) == set(built.EXPORTS) | {"gmq_status_string", "gmq_last_cuda_error"}


def test_seed_genz_matches_input_module(built):
    for fam, S in G.GENZ_TARGET_SUM.items():
        for d in (1, 3, 8, 12):
            for seed in (1, 7, 2511):
                a, u = built.seed_genz(seed, fam, d, S)
                a2, u2 = G.seed_genz(seed, fam, d, S)
                assert np.array_equal(a, a2) and np.array_equal(u, u2)
                assert abs(a.sum() - S) < 1e-12 * S


def test_splitmix64_reference_values():
    # first outputs of SplitMix64 seeded with 0 (published test vector of the
    # generator's reference implementation)
    g = G.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                0x06C45D188009454F]


def test_host_only_calls(built):
    assert built.status_string(0) == "converged"
    assert built.status_string(-4) == "non-finite integrand value"
    o = built.default_options()
    assert o.rel_tol == 1e-6 and o.abs_tol == 1e-16 and o.max_regions == 1 << 22
    b8 = built.pool_bytes(8, 1 << 24)
    # two region lists of 2 * 8 doubles per region dominate
    assert 2 * 16 * 8 * (1 << 24) < b8 < 2 * 16 * 8 * (1 << 24) * 1.2
    with pytest.raises(built.GmqError):
        built.pool_bytes(0, 10)
    with pytest.raises(built.GmqError):
        built.seed_genz(1, 0, 0, 1.0)
