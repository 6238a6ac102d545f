"""Python binding of the C ABI in ``include/gmq.h`` (ctypes).

Argument marshalling only: every step of the quadrature runs in the CUDA
library.  PyTorch supplies device memory (tensors) and the current stream.
The names follow the C calls without the ``gmq_`` prefix.  If the library
has not been built the import fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libgmq.so")

MAX_DIM = 16

OK, CAP_REACHED, MAX_ITERS, ROUNDOFF_LIMIT = 0, 1, 2, 3
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT = -1, -2, -3, -4, -5

(OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS,
 POLY_SUMSQ11) = range(7)
FP64, MIXED = 0, 1
VOLUME_SHARE, LOCAL_REL = 0, 1
EST_EMBEDDED, EST_NULL_RULES = 0, 1
EVAL_SEPARABLE, EVAL_NODEWISE = 0, 1

_dp = C.POINTER(C.c_double)


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("family", C.c_int32), ("lo", _dp), ("hi", _dp),
                ("a", _dp), ("u", _dp)]


class Options(C.Structure):
    _fields_ = [("rel_tol", C.c_double), ("abs_tol", C.c_double), ("max_regions", C.c_int64),
                ("init_splits", C.c_int32), ("max_iters", C.c_int32), ("precision", C.c_int32),
                ("classifier", C.c_int32), ("lanes", C.c_int32), ("flags", C.c_int32),
                ("rule", C.c_int32), ("estimator", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("integral", C.c_double), ("error", C.c_double),
                ("regions_evaluated", C.c_int64), ("function_evals", C.c_int64),
                ("final_active", C.c_int64), ("iterations", C.c_int32), ("status", C.c_int32)]


class KernelStats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("regions", C.c_int64), ("ms", C.c_double)]


KERNELS = ("rule", "sum", "classify", "split", "partition")


class Sweep(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_split", C.c_int64), ("I", C.c_double), ("E", C.c_double),
                ("I_ret", C.c_double), ("E_ret", C.c_double), ("budget", C.c_double)]


EXPORTS = ("gmq_create", "gmq_destroy", "gmq_set_stream", "gmq_set_pool", "gmq_pool_bytes",
           "gmq_default_options", "gmq_integrate", "gmq_last_trace", "gmq_seed_genz",
           "gmq_status_string", "gmq_launch_count", "gmq_eval_rule", "gmq_classify_split",
           "gmq_tree_sum", "gmq_partition", "gmq_profile_enable", "gmq_profile_reset",
           "gmq_profile_read", "gmq_tree_sum_noalloc", "gmq_partition_copy", "gmq_rule_grad",
           "gmq_integrate_batch", "gmq_last_batch_info", "gmq_eval_rule_gk", "gmq_gk_table",
           "gmq_math_exp", "gmq_math_rcp", "gmq_math_cos", "gmq_probe_fp_rate", "gmq_null_rule_table",
           "gmq_set_eval_mode")

KEEP_PARTITION = 1
BATCH_HOST_LOOP = 2
RULE_GENZ_MALIK = 0
RULE_GAUSS_KRONROD = 1
GK_MAX_DIM = 6


class BatchInfo(C.Structure):
    _fields_ = [("rule_block", C.c_int32), ("rule_grid", C.c_int32), ("sweeps", C.c_int32),
                ("used_graph", C.c_int32), ("autotuned", C.c_int32), ("pauses", C.c_int32),
                ("evictions", C.c_int32), ("forced_lanes", C.c_int32),
                ("lanes_t1", C.c_int64), ("lanes_t4", C.c_int64), ("lanes_t32", C.c_int64),
                ("lane_sweeps", C.c_int32 * 4),
                ("tune_n", C.c_int64 * 5), ("tune_ms", (C.c_double * 4) * 5),
                ("rule_regions", C.c_int64), ("carried_regions", C.c_int64),
                ("list_regions", C.c_int64)]

ERR_TOO_LARGE = -6
NOALLOC_MAX_N = 1 << 23


def null_rule_table(dim: int):
    """The library's null-rule weights for dimension dim (4 x 5: rows N1..N4,
    columns the node classes; unit volume)."""
    out = np.zeros(20)
    _check("gmq_null_rule_table", lib().gmq_null_rule_table(dim, out.ctypes.data_as(_dp)))
    return out.reshape(4, 5)


def gk_table():
    """The library's 1-D Gauss-Kronrod tables (45 floats: nodes, K15 and G7
    weights)."""
    import numpy as np
    out = np.zeros(45)
    _check("gmq_gk_table", lib().gmq_gk_table(out.ctypes.data_as(_dp)))
    return out


class GmqError(RuntimeError):
    def __init__(self, call, code):
        self.code = code
        extra = ""
        if code in (ERR_CUDA, ERR_OOM):
            extra = f" [{lib().gmq_last_cuda_error().decode()}]"
        super().__init__(f"{call} failed: {status_string(code)} ({code}){extra}")


_lib = None


def lib():
    """Load the library (ctypes); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing "
                          "(run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "gmq_create": [C.POINTER(vp), C.c_int, C.c_size_t],
        "gmq_destroy": [vp],
        "gmq_set_stream": [vp, vp],
        "gmq_set_pool": [vp, vp, C.c_size_t],
        "gmq_set_eval_mode": [vp, C.c_int32],
        "gmq_pool_bytes": [i32, i64, i32, C.POINTER(C.c_size_t)],
        "gmq_default_options": [C.POINTER(Options)],
        "gmq_integrate": [vp, C.POINTER(Problem), C.POINTER(Options), C.POINTER(Result)],
        "gmq_last_trace": [vp, C.POINTER(Sweep), i32, C.POINTER(i32)],
        "gmq_seed_genz": [C.c_uint64, i32, i32, dbl, _dp, _dp],
        "gmq_launch_count": [vp, C.POINTER(i64)],
        "gmq_eval_rule": [vp, C.POINTER(Problem), i32, i32, i32, i64, vp, vp, i64, vp, vp, vp,
                          vp],
        "gmq_classify_split": [vp, i32, i64, vp, vp, i64, vp, vp, vp, vp, dbl, dbl, i32, vp, vp,
                               i64, i64, vp, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl)],
        "gmq_tree_sum": [vp, i64, vp, C.POINTER(dbl)],
        "gmq_partition": [vp, i32, _dp, _dp, i32, vp, vp, i64],
        "gmq_profile_enable": [vp, i32],
        "gmq_profile_reset": [vp],
        "gmq_profile_read": [vp, i32, C.POINTER(KernelStats)],
        "gmq_tree_sum_noalloc": [i32, i64, vp, vp, vp],
        "gmq_partition_copy": [vp, vp, vp, i64, i64, C.POINTER(i64)],
        "gmq_rule_grad": [vp, C.POINTER(Problem), i64, vp, vp, i64, C.POINTER(dbl), _dp],
        "gmq_integrate_batch": [vp, i32, C.POINTER(Problem), _dp, C.POINTER(Options), i64,
                                C.POINTER(Result)],
        "gmq_last_batch_info": [vp, C.POINTER(BatchInfo)],
        "gmq_eval_rule_gk": [vp, C.POINTER(Problem), i64, vp, vp, i64, vp, vp, vp, vp],
        "gmq_gk_table": [_dp],
        "gmq_null_rule_table": [i32, _dp],
        "gmq_math_exp": [vp, i64, vp, vp],
        "gmq_math_rcp": [vp, i64, vp, vp],
        "gmq_math_cos": [vp, i64, vp, vp],
        "gmq_probe_fp_rate": [vp, i32, i32, i64, C.POINTER(dbl), C.POINTER(dbl)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.gmq_status_string.argtypes = [C.c_int]
    L.gmq_status_string.restype = C.c_char_p
    L.gmq_last_cuda_error.argtypes = []
    L.gmq_last_cuda_error.restype = C.c_char_p
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().gmq_status_string(int(code)).decode()


def _check(call, code, ok=(OK,)):
    if code not in ok:
        raise GmqError(call, code)
    return code


def _f64(x, d=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if d is not None and a.shape != (d,):
        raise ValueError(f"expected {d} values, got shape {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp)


def pool_bytes(dim: int, max_regions: int, flags: int = 0) -> int:
    out = C.c_size_t()
    _check("gmq_pool_bytes", lib().gmq_pool_bytes(dim, max_regions, flags, C.byref(out)))
    return int(out.value)


def default_options() -> Options:
    o = Options()
    _check("gmq_default_options", lib().gmq_default_options(C.byref(o)))
    return o


def seed_genz(seed: int, family: int, dim: int, target_sum: float):
    a = np.zeros(dim)
    u = np.zeros(dim)
    _check("gmq_seed_genz", lib().gmq_seed_genz(seed, family, dim, target_sum, _ptr(a), _ptr(u)))
    return a, u


def tree_sum_noalloc(v, out, stream=None) -> int:
    """Enqueue the allocation-free pairwise sum of the CUDA float64 tensor v
    into the one-element CUDA float64 tensor out, on `stream` (default: the
    current torch stream of v's device).  Returns the status code; the
    value is in `out` once the stream gets there.  Calls whose GPU work
    overlaps share one scratch array and race."""
    import torch
    if not (v.is_cuda and v.dtype == torch.float64 and out.is_cuda and out.dtype == torch.float64):
        raise ValueError("expected CUDA float64 tensors")
    if v.numel() > 1 and not v.is_contiguous():
        raise ValueError("v must be contiguous")
    dev = v.device.index
    if out.device != v.device:
        raise ValueError(f"out is on {out.device}, v on {v.device}")
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    if s.device != v.device:
        raise ValueError(f"stream is on {s.device}, v on {v.device}")
    return lib().gmq_tree_sum_noalloc(dev, v.numel(), C.c_void_p(v.data_ptr()),
                                      C.c_void_p(out.data_ptr()), C.c_void_p(s.cuda_stream))


@dataclass
class IntegrateResult:
    integral: float
    error: float
    regions_evaluated: int
    function_evals: int
    final_active: int
    iterations: int
    status: int

    @property
    def status_str(self) -> str:
        return status_string(self.status)


class _ProblemHandle:
    def __init__(self, family, a, u, lo, hi, dim=None):
        d = dim if dim is not None else len(np.atleast_1d(a))
        self.a = _f64(np.zeros(d) if a is None else a, d)
        self.u = _f64(np.zeros(d) if u is None else u, d)
        self.lo = _f64(np.zeros(d) if lo is None else lo, d)
        self.hi = _f64(np.ones(d) if hi is None else hi, d)
        self.s = Problem(d, int(family), _ptr(self.lo), _ptr(self.hi), _ptr(self.a), _ptr(self.u))


def _dptr(t):
    return C.c_void_p(t.data_ptr())


class Context:
    """One library context on one CUDA device; runs on torch's current stream
    of that device unless ``set_stream`` says otherwise."""

    def __init__(self, device: int = 0, pool_bytes_hint: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        h = C.c_void_p()
        _check("gmq_create", lib().gmq_create(C.byref(h), device, pool_bytes_hint))
        self.h = h
        self.set_stream(stream if stream is not None else torch.cuda.current_stream(device))

    def set_stream(self, stream):
        self.stream = stream
        _check("gmq_set_stream", lib().gmq_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def set_pool(self, tensor):
        """Use a caller-owned uint8 CUDA tensor as the region pool (None to undo)."""
        self._pool = tensor
        if tensor is None:
            _check("gmq_set_pool", lib().gmq_set_pool(self.h, None, 0))
        else:
            _check("gmq_set_pool", lib().gmq_set_pool(self.h, _dptr(tensor), tensor.numel()))

    def set_eval_mode(self, mode):
        """How the FP64 Genz-Malik kernels evaluate f at the nodes:
        EVAL_SEPARABLE (per-axis terms once per region, the default) or
        EVAL_NODEWISE (f from every node's coordinates)."""
        _check("gmq_set_eval_mode", lib().gmq_set_eval_mode(self.h, int(mode)))

    def close(self):
        if getattr(self, "h", None):
            lib().gmq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, on: bool = True):
        """Time every kernel launch with CUDA events on the context stream."""
        _check("gmq_profile_enable", lib().gmq_profile_enable(self.h, 1 if on else 0))

    def profile_reset(self):
        _check("gmq_profile_reset", lib().gmq_profile_reset(self.h))

    def profile_read(self):
        out = {}
        for k, name in enumerate(KERNELS):
            s = KernelStats()
            _check("gmq_profile_read", lib().gmq_profile_read(self.h, k, C.byref(s)))
            out[name] = {"launches": int(s.launches), "regions": int(s.regions), "ms": s.ms}
        return out

    PROBE_OPS = ("fma", "add", "mul")

    def probe_fp_rate(self, precision=FP64, op="fma", iters=None):
        """Measured issue rate of one floating-point operation on this GPU
        (lane operations per second) and the probe launch's milliseconds;
        FP64 by default, FP32 with MIXED; op "fma", "add" or "mul"."""
        if iters is None:
            iters = 20000 if precision == FP64 else 1_000_000
        rate = C.c_double()
        ms = C.c_double()
        _check("gmq_probe_fp_rate", lib().gmq_probe_fp_rate(
            self.h, precision, self.PROBE_OPS.index(op), iters, C.byref(rate), C.byref(ms)))
        return rate.value, ms.value

    def launch_count(self) -> int:
        n = C.c_int64()
        _check("gmq_launch_count", lib().gmq_launch_count(self.h, C.byref(n)))
        return int(n.value)

    def integrate(self, family, a=None, u=None, rel_tol=1e-6, lo=None, hi=None, abs_tol=1e-16,
                  max_regions=1 << 22, init_splits=0, max_iters=0, precision=FP64,
                  classifier=VOLUME_SHARE, lanes=0, dim=None, check=True,
                  keep_partition=False, rule=RULE_GENZ_MALIK,
                  estimator=EST_EMBEDDED) -> IntegrateResult:
        p = _ProblemHandle(family, a, u, lo, hi, dim)
        o = Options(rel_tol, abs_tol, max_regions, init_splits, max_iters, precision, classifier,
                    lanes, KEEP_PARTITION if keep_partition else 0, rule, estimator)
        r = Result()
        self._last_dim = p.s.dim
        code = lib().gmq_integrate(self.h, C.byref(p.s), C.byref(o), C.byref(r))
        if check:
            _check("gmq_integrate", code, ok=(OK, CAP_REACHED, MAX_ITERS, ROUNDOFF_LIMIT))
        return IntegrateResult(r.integral, r.error, r.regions_evaluated, r.function_evals,
                               r.final_active, r.iterations, code)

    def integrate_batch(self, problems, rel_tols=None, max_regions=1 << 24, abs_tol=1e-16,
                        init_splits=0, max_iters=0, classifier=VOLUME_SHARE, host_loop=False,
                        pool_regions=0, lanes=0, precision=FP64, estimator=EST_EMBEDDED):
        """Integrate many problems in one device-resident loop.  problems:
        objects with family, dim, a, u (and optional lo, hi, rel_tol).
        max_regions is each problem's cap, pool_regions the shared pool (0:
        the library's default); lanes 1, 4, 32 or 128 fixes the rule
        kernel's lanes per region (0: autotuned per sweep; MIXED runs one lane
        per region).  Returns one IntegrateResult per problem."""
        hs = [_ProblemHandle(p.family, p.a, p.u, getattr(p, "lo", None), getattr(p, "hi", None),
                             p.dim) for p in problems]
        arr = (Problem * len(hs))(*[h.s for h in hs])
        if rel_tols is None:
            rel_tols = [p.rel_tol for p in problems]
        tols = _f64(rel_tols, len(hs))
        o = Options(0.0, abs_tol, max_regions, init_splits, max_iters, precision, classifier, lanes,
                    BATCH_HOST_LOOP if host_loop else 0, RULE_GENZ_MALIK, estimator)
        res = (Result * len(hs))()
        _check("gmq_integrate_batch", lib().gmq_integrate_batch(self.h, len(hs), arr, _ptr(tols),
                                                                C.byref(o), pool_regions, res))
        return [IntegrateResult(r.integral, r.error, r.regions_evaluated, r.function_evals,
                                r.final_active, r.iterations, r.status) for r in res]

    def last_batch_info(self):
        info = BatchInfo()
        _check("gmq_last_batch_info", lib().gmq_last_batch_info(self.h, C.byref(info)))
        return {"rule_block": info.rule_block, "rule_grid": info.rule_grid,
                "sweeps": info.sweeps, "used_graph": bool(info.used_graph),
                "autotuned": bool(info.autotuned), "pauses": int(info.pauses),
                "evictions": int(info.evictions), "forced_lanes": int(info.forced_lanes),
                "lanes_t1": int(info.lanes_t1), "lanes_t4": int(info.lanes_t4),
                "lanes_t32": int(info.lanes_t32),
                "lane_sweeps": list(info.lane_sweeps),
                "rule_regions": int(info.rule_regions),
                "carried_regions": int(info.carried_regions),
                "list_regions": int(info.list_regions),
                "tune": [{"n": int(info.tune_n[i]), "ms": list(info.tune_ms[i])}
                         for i in range(5) if info.tune_n[i] > 0]}

    def partition_copy(self):
        """The final partition of the last integrate(keep_partition=True) call
        as CUDA float64 tensors (center, halfw) of shape [dim, count]."""
        torch = self.torch
        cnt = C.c_int64()
        _check("gmq_partition_copy", lib().gmq_partition_copy(self.h, None, None, 0, 0,
                                                              C.byref(cnt)))
        n = int(cnt.value)
        if n < 0:
            raise RuntimeError("no partition was kept by the last integration")
        return self._copy_partition(n)

    def _copy_partition(self, n):
        torch = self.torch
        # the dimension is that of the last problem; recover it from the pool copy
        d = self._last_dim
        c = torch.empty((d, max(n, 1)), dtype=torch.float64, device=f"cuda:{self.device}")
        h = torch.empty_like(c)
        cnt = C.c_int64()
        _check("gmq_partition_copy", lib().gmq_partition_copy(self.h, _dptr(c), _dptr(h),
                                                              max(n, 1), n, C.byref(cnt)))
        return c[:, :n], h[:, :n]

    def rule_grad(self, family, a, u, center, halfw, lo=None, hi=None):
        """Frozen-partition quadrature Q and dQ/d(a_1..a_d, u_1..u_d) over the
        regions (center, halfw: CUDA float64 [dim, n]).  Returns (grad, Q)."""
        d, n = center.shape
        ld = self._ld(center, halfw) if n > 0 else 1
        p = _ProblemHandle(family, a, u, lo, hi, d)
        g = np.zeros(2 * d)
        q = C.c_double()
        _check("gmq_rule_grad", lib().gmq_rule_grad(self.h, C.byref(p.s), n, _dptr(center),
                                                    _dptr(halfw), ld, C.byref(q), _ptr(g)))
        return g, q.value

    def last_trace(self):
        cnt = C.c_int32()
        lib().gmq_last_trace(self.h, None, 0, C.byref(cnt))
        arr = (Sweep * max(1, cnt.value))()
        _check("gmq_last_trace", lib().gmq_last_trace(self.h, arr, cnt.value, C.byref(cnt)))
        return [dict(n=s.n, n_split=s.n_split, I=s.I, E=s.E, I_ret=s.I_ret, E_ret=s.E_ret,
                     budget=s.budget) for s in arr[:cnt.value]]

    # ---- step-level calls on torch CUDA tensors -------------------------

    @staticmethod
    def _ld(center, halfw):
        """Leading dimension of a [dim, n] pair with unit stride along regions
        (the stride of a size-1 dimension is not meaningful)."""
        d, n = center.shape
        if halfw.shape != center.shape:
            raise ValueError("center and halfw must have the same shape [dim, n]")
        for t in (center, halfw):
            if n > 1 and t.stride(1) != 1:
                raise ValueError("regions must be contiguous along the last dimension")
        if d == 1:
            return max(n, 1)
        if halfw.stride(0) != center.stride(0) or center.stride(0) < n:
            raise ValueError("center and halfw must share a row stride >= n")
        return center.stride(0)

    def _dev(self, t, dtype):
        torch = self.torch
        if not (t.is_cuda and t.dtype == dtype):
            raise ValueError(f"expected a CUDA {dtype} tensor")
        return t

    def eval_rule(self, family, a, u, center, halfw, lo=None, hi=None, precision=FP64, lanes=0,
                  estimator=EST_EMBEDDED):
        """center, halfw: CUDA float64 tensors [dim, n] with unit stride along
        regions.  Returns (I7, err, volfrac, axis) tensors of length n."""
        torch = self.torch
        center = self._dev(center, torch.float64)
        halfw = self._dev(halfw, torch.float64)
        d, n = center.shape
        ld = self._ld(center, halfw)
        p = _ProblemHandle(family, a, u, lo, hi, d)
        dev = center.device
        i7 = torch.empty(n, dtype=torch.float64, device=dev)
        err = torch.empty(n, dtype=torch.float64, device=dev)
        vf = torch.empty(n, dtype=torch.float64, device=dev)
        ax = torch.empty(n, dtype=torch.uint8, device=dev)
        _check("gmq_eval_rule", lib().gmq_eval_rule(
            self.h, C.byref(p.s), precision, lanes, estimator, n, _dptr(center), _dptr(halfw),
            ld, _dptr(i7), _dptr(err), _dptr(vf), _dptr(ax)))
        return i7, err, vf, ax

    def eval_rule_gk(self, family, a, u, center, halfw, lo=None, hi=None):
        """The tensor-product Gauss-Kronrod rule; arguments and results as
        for eval_rule (I_K in place of I7)."""
        torch = self.torch
        center = self._dev(center, torch.float64)
        halfw = self._dev(halfw, torch.float64)
        d, n = center.shape
        ld = self._ld(center, halfw)
        p = _ProblemHandle(family, a, u, lo, hi, d)
        dev = center.device
        ik = torch.empty(n, dtype=torch.float64, device=dev)
        err = torch.empty(n, dtype=torch.float64, device=dev)
        vf = torch.empty(n, dtype=torch.float64, device=dev)
        ax = torch.empty(n, dtype=torch.uint8, device=dev)
        _check("gmq_eval_rule_gk", lib().gmq_eval_rule_gk(
            self.h, C.byref(p.s), n, _dptr(center), _dptr(halfw), ld, _dptr(ik), _dptr(err),
            _dptr(vf), _dptr(ax)))
        return ik, err, vf, ax

    def math_exp(self, x):
        """The library's FP64 exponential on a CUDA float64 tensor."""
        torch = self.torch
        x = self._dev(x, torch.float64).contiguous()
        y = torch.empty_like(x)
        _check("gmq_math_exp", lib().gmq_math_exp(self.h, x.numel(), _dptr(x), _dptr(y)))
        return y

    def math_rcp(self, x):
        """The library's FP64 reciprocal on a CUDA float64 tensor."""
        torch = self.torch
        x = self._dev(x, torch.float64).contiguous()
        y = torch.empty_like(x)
        _check("gmq_math_rcp", lib().gmq_math_rcp(self.h, x.numel(), _dptr(x), _dptr(y)))
        return y

    def math_cos(self, x):
        """The library's FP64 cosine on a CUDA float64 tensor."""
        torch = self.torch
        x = self._dev(x, torch.float64).contiguous()
        y = torch.empty_like(x)
        _check("gmq_math_cos", lib().gmq_math_cos(self.h, x.numel(), _dptr(x), _dptr(y)))
        return y

    def classify_split(self, center, halfw, i7, err, volfrac, axis, budget, rel_tol=0.0,
                       classifier=VOLUME_SHARE, cap_out=None):
        torch = self.torch
        d, n = center.shape
        ld = self._ld(center, halfw)
        cap = 2 * n if cap_out is None else cap_out
        dev = center.device
        co = torch.zeros((d, max(cap, 1)), dtype=torch.float64, device=dev)
        ho = torch.zeros((d, max(cap, 1)), dtype=torch.float64, device=dev)
        flags = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
        ns = C.c_int64()
        ri = C.c_double()
        re_ = C.c_double()
        code = lib().gmq_classify_split(
            self.h, d, n, _dptr(center), _dptr(halfw), ld, _dptr(i7), _dptr(err),
            _dptr(volfrac) if volfrac is not None else None, _dptr(axis), budget, rel_tol,
            classifier, _dptr(co), _dptr(ho), max(cap, 1), cap, _dptr(flags), C.byref(ns),
            C.byref(ri), C.byref(re_))
        _check("gmq_classify_split", code, ok=(OK, CAP_REACHED))
        k = int(ns.value)
        return dict(status=code, n_split=k, ret_i=ri.value, ret_e=re_.value, flags=flags[:n],
                    center=co[:, :2 * k], halfw=ho[:, :2 * k])

    def tree_sum(self, v) -> float:
        v = self._dev(v, self.torch.float64).contiguous()
        out = C.c_double()
        _check("gmq_tree_sum", lib().gmq_tree_sum(self.h, v.numel(), _dptr(v), C.byref(out)))
        return out.value

    def partition(self, dim, s, lo=None, hi=None):
        torch = self.torch
        lo = _f64(np.zeros(dim) if lo is None else lo, dim)
        hi = _f64(np.ones(dim) if hi is None else hi, dim)
        n = s ** dim
        c = torch.empty((dim, n), dtype=torch.float64, device=f"cuda:{self.device}")
        h = torch.empty_like(c)
        _check("gmq_partition", lib().gmq_partition(self.h, dim, _ptr(lo), _ptr(hi), s, _dptr(c),
                                                     _dptr(h), n))
        return c, h
