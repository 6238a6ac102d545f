"""gmq_tree_sum_noalloc: the allocation-free pairwise sum, for callers that
cannot allocate device memory where they need a sum (their memory belongs to
their own allocator or a fixed start-up budget, or they cannot take the
device-wide synchronisation of cudaMalloc/cudaFree).  Its scratch is a
static device array, so this file runs last: if it fails, a run that stops
at the first failure has already run every other test.  It must pass on its
own in a fresh process as well as after the rest of the suite.

Checked through the C ABI against gmq_tree_sum (which allocates its scratch
through the context) with the tolerance the tree-sum tests use: none, the
two calls use the same summation tree.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc_sum(gmq, v):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=v.device)
    code = gmq.tree_sum_noalloc(v, out)
    assert code == gmq.OK, gmq.status_string(code)
    torch.cuda.current_stream(v.device).synchronize()
    return float(out.item())


def test_noalloc_sum_matches_tree_sum_twice_in_a_row(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    rng = np.random.default_rng(20251103)
    # two calls in a row on different inputs: the second must not see the
    # first call's partial sums or ticket
    for n in (3_000_001, 1025):
        v = torch.tensor(rng.standard_normal(n) * np.exp(rng.uniform(-20, 20, n)),
                         device="cuda")
        want = gpu_ctx.tree_sum(v)
        got = _noalloc_sum(gmq, v)
        assert got == want, (n, got, want)
    # and the same input twice
    v = torch.tensor(rng.uniform(-1, 1, 1 << 20), device="cuda")
    a = _noalloc_sum(gmq, v)
    b = _noalloc_sum(gmq, v)
    assert a == b == gpu_ctx.tree_sum(v)


def test_noalloc_sum_limits(gpu_ctx):
    from paper_2511_01573_gb300 import gmq
    # the largest accepted length, then one more: rejected with a clear code
    v = torch.ones(gmq.NOALLOC_MAX_N + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert gmq.tree_sum_noalloc(v, out) == gmq.ERR_TOO_LARGE
    assert "scratch" in gmq.status_string(gmq.ERR_TOO_LARGE)
    assert _noalloc_sum(gmq, v[:gmq.NOALLOC_MAX_N]) == float(gmq.NOALLOC_MAX_N)
    assert _noalloc_sum(gmq, v[:0]) == 0.0
    assert _noalloc_sum(gmq, v[:1]) == 1.0


def test_noalloc_sum_on_a_side_stream_and_another_thread(gpu_ctx):
    """The call orders its own clear and launch on the stream it is given:
    on a fresh side stream, with nothing synchronising the default stream,
    it still gives the bits of gmq_tree_sum; a later call from another host
    thread (after the first has finished) does too."""
    import threading
    from paper_2511_01573_gb300 import gmq
    rng = np.random.default_rng(7)
    v = torch.tensor(rng.standard_normal(2_000_003), device="cuda")
    want = gpu_ctx.tree_sum(v)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    assert gmq.tree_sum_noalloc(v, out, stream=side) == gmq.OK
    side.synchronize()
    assert float(out.item()) == want
    res = {}

    def worker():
        o = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        res["code"] = gmq.tree_sum_noalloc(v, o, stream=side)
        side.synchronize()
        res["sum"] = float(o.item())

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert res["code"] == gmq.OK and res["sum"] == want


def test_noalloc_sum_rejects_host_memory(gpu_ctx):
    """Pointers that are not device memory of the given device are refused
    before anything is enqueued (a pinned host result buffer here)."""
    import ctypes
    from paper_2511_01573_gb300 import gmq
    v = torch.ones(1000, dtype=torch.float64, device="cuda")
    host = torch.full((1,), 5.0, dtype=torch.float64).pin_memory()
    code = gmq.lib().gmq_tree_sum_noalloc(0, v.numel(), ctypes.c_void_p(v.data_ptr()),
                                          ctypes.c_void_p(host.data_ptr()), None)
    assert code == gmq.ERR_INVALID and float(host[0]) == 5.0
