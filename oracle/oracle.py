"""ctypes wrapper of the plain FP64 CPU oracle (``gm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  ``build()`` compiles the
C source with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gm_oracle.c")
HDR = os.path.join(HERE, "gm_oracle.h")
LIB = os.path.join(HERE, "_build", "libgm_oracle.so")

_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)
INTEGRAND = C.CFUNCTYPE(C.c_double, _dp, C.c_int, C.c_void_p)


class Family(C.Structure):
    _fields_ = [("family", C.c_int32), ("d", C.c_int32), ("a", _dp), ("u", _dp)]


class RuleOut(C.Structure):
    _fields_ = [("i7", C.c_double), ("i5", C.c_double), ("err", C.c_double),
                ("s", C.c_double * 5), ("sabs", C.c_double * 5), ("vol", C.c_double),
                ("f0", C.c_double), ("axis", C.c_int32), ("axis_tie", C.c_int32),
                ("flat", C.c_int32), ("split_bad", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("rel_tol", C.c_double), ("abs_tol", C.c_double), ("max_regions", C.c_int64),
                ("init_splits", C.c_int32), ("max_iters", C.c_int32), ("classifier", C.c_int32),
                ("rule", C.c_int32), ("gk", _dp), ("estimator", C.c_int32), ("null_w", _dp)]


class NullOut(C.Structure):
    _fields_ = [("nul", C.c_double * 4), ("e", C.c_double * 3), ("r", C.c_double),
                ("est", C.c_double), ("est_alt", C.c_double), ("noise", C.c_double),
                ("band", C.c_double), ("regime", C.c_int32), ("regime_tie", C.c_int32)]


class GkOut(C.Structure):
    _fields_ = [("ik", C.c_double), ("ig", C.c_double), ("err", C.c_double),
                ("vol", C.c_double), ("scale", C.c_double), ("axis", C.c_int32),
                ("axis_tie", C.c_int32), ("flat", C.c_int32), ("split_bad", C.c_int32)]


RULE_GM = 0
RULE_GK = 1
EST_EMBEDDED = 0
EST_NULL_RULES = 1
_GK = None
_NULL = {}


def null_table(d: int):
    """The 4 x 5 null-rule weight table for dimension d (oracle/null_rules.py,
    exact rational arithmetic, rounded once)."""
    if d not in _NULL:
        from oracle.null_rules import null_table as nt
        _NULL[d] = np.ascontiguousarray(np.array(nt(d), dtype=np.float64))
    return _NULL[d]


def gk_table():
    """The 45-double Gauss-Kronrod table (nodes, K15 weights, G7 weights)
    from gk_tables (exact rational arithmetic, rounded)."""
    global _GK
    if _GK is None:
        from oracle.gk_tables import gk15_float
        x, wk, wg = gk15_float()
        _GK = np.ascontiguousarray(np.array(x + wk + wg, dtype=np.float64))
    return _GK


def _options(rel_tol, abs_tol, max_regions, init_splits, max_iters, classifier, rule,
             estimator=EST_EMBEDDED, d=None):
    gk = gk_table() if rule == RULE_GK else None
    nw = null_table(d) if estimator == EST_NULL_RULES else None
    o = Options(rel_tol, abs_tol, max_regions, init_splits, max_iters, classifier, rule,
                _p(gk) if gk is not None else None, estimator,
                _p(nw) if nw is not None else None)
    o._keep = (gk, nw)
    return o


class Result(C.Structure):
    _fields_ = [("integral", C.c_double), ("error", C.c_double),
                ("regions_evaluated", C.c_int64), ("function_evals", C.c_int64),
                ("final_active", C.c_int64), ("iterations", C.c_int32), ("status", C.c_int32),
                ("near_ties", C.c_int64)]


class Trace(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_split", C.c_int64), ("near_ties", C.c_int64),
                ("I", C.c_double), ("E", C.c_double), ("I_ret", C.c_double),
                ("E_ret", C.c_double), ("budget", C.c_double)]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    stale = (not os.path.exists(LIB) or
             os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(HDR)))
    if force or stale:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        L.or_num_nodes.restype = C.c_int64
        L.or_num_nodes.argtypes = [C.c_int]
        L.or_lambdas.argtypes = [_dp]
        L.or_weights.argtypes = [C.c_int, _dp, _dp]
        L.or_family_eval.restype = C.c_double
        L.or_family_eval.argtypes = [_dp, C.c_int, C.c_void_p]
        L.or_rule.argtypes = [C.c_int, _dp, _dp, C.c_void_p, C.c_void_p, _dp, C.POINTER(RuleOut)]
        L.or_rule_regions.argtypes = [C.POINTER(Family), C.c_int64, _dp, _dp, _dp, _dp, _dp, _dp,
                                      _i32p, _i32p, _i32p, _dp]
        L.or_pairwise_sum.restype = C.c_double
        L.or_pairwise_sum.argtypes = [_dp, C.c_int64]
        L.or_auto_splits.restype = C.c_int32
        L.or_auto_splits.argtypes = [C.c_int, C.c_int64]
        L.or_partition.restype = C.c_int64
        L.or_partition.argtypes = [C.c_int, _dp, _dp, C.c_int32, _dp, _dp]
        L.or_classify.restype = C.c_int64
        L.or_classify.argtypes = [C.c_int, C.c_int64, _dp, _dp, _dp, _i32p, _dp, C.c_double,
                                  C.c_double, C.c_double, C.c_int32, _u8p, _dp, _dp,
                                  C.POINTER(C.c_int64)]
        L.or_bisect.restype = C.c_int64
        L.or_bisect.argtypes = [C.c_int, C.c_int64, _dp, _dp, _i32p, _u8p, _dp, _dp]
        L.or_gk_nodes.restype = C.c_int64
        L.or_gk_nodes.argtypes = [C.c_int]
        L.or_rule_gk.argtypes = [C.c_int, _dp, _dp, C.c_void_p, C.c_void_p, _dp, _dp,
                                 C.POINTER(GkOut)]
        L.or_rule_gk_regions.argtypes = [C.POINTER(Family), C.c_int64, _dp, _dp, _dp, _dp, _dp,
                                         _dp, _dp, _i32p, _i32p, _i32p, _dp]
        L.or_null_estimate.argtypes = [C.POINTER(RuleOut), _dp, C.POINTER(NullOut)]
        L.or_rule_regions_est.argtypes = [C.POINTER(Family), C.c_int64, _dp, _dp, _dp, _dp, _dp,
                                          _dp, _i32p, _i32p, _i32p, _dp, _dp, _dp]
        L.or_classify_band.restype = C.c_int64
        L.or_classify_band.argtypes = [C.c_int, C.c_int64, _dp, _dp, _dp, _i32p, _dp, _dp,
                                       C.c_double, C.c_double, C.c_double, C.c_int32, _u8p, _dp,
                                       _dp, C.POINTER(C.c_int64)]
        L.or_integrate.restype = C.c_int32
        L.or_integrate.argtypes = [C.POINTER(Family), _dp, _dp, C.POINTER(Options),
                                   C.POINTER(Result), C.POINTER(Trace), C.c_int32]
        _lib = L
    return _lib


def _p(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_nodes(d: int) -> int:
    return int(lib().or_num_nodes(d))


def lambdas():
    out = np.zeros(4)
    lib().or_lambdas(_p(out))
    return out


def weights(d: int):
    w7 = np.zeros(5)
    w5 = np.zeros(5)
    lib().or_weights(d, _p(w7), _p(w5))
    return w7, w5


class _FamilyHandle:
    """Keeps the parameter arrays alive while C holds pointers to them."""

    def __init__(self, family: int, a, u):
        self.a = _f64(a)
        self.u = _f64(u)
        self.s = Family(int(family), len(self.a), _p(self.a), _p(self.u))


def family_eval(family: int, a, u, x) -> float:
    fh = _FamilyHandle(family, a, u)
    x = _f64(x)
    return float(lib().or_family_eval(_p(x), len(x), C.cast(C.pointer(fh.s), C.c_void_p)))


@dataclass
class Rule:
    i7: float
    i5: float
    err: float
    s: np.ndarray
    sabs: np.ndarray
    vol: float
    f0: float
    axis: int
    axis_tie: bool
    flat: bool
    split_bad: bool
    D: np.ndarray


def rule(c, h, f=None, family=None, a=None, u=None) -> Rule:
    """Rule on one region; f is a Python callable f(x: ndarray) -> float, or a
    built-in family with parameters a, u."""
    c = _f64(c)
    h = _f64(h)
    d = len(c)
    D = np.zeros(d)
    out = RuleOut()
    if f is not None:
        def cb(xp, dd, _ctx):
            return float(f(np.ctypeslib.as_array(xp, shape=(dd,)).copy()))
        cfun = INTEGRAND(cb)
        lib().or_rule(d, _p(c), _p(h), C.cast(cfun, C.c_void_p), None, _p(D), C.byref(out))
    else:
        fh = _FamilyHandle(family, a, u)
        fn = C.cast(lib().or_family_eval, C.c_void_p)
        lib().or_rule(d, _p(c), _p(h), fn, C.cast(C.pointer(fh.s), C.c_void_p), _p(D),
                      C.byref(out))
    r = Rule(out.i7, out.i5, out.err, np.array(out.s[:]), np.array(out.sabs[:]), out.vol,
             out.f0, out.axis, bool(out.axis_tie), bool(out.flat), bool(out.split_bad), D)
    r._raw = out
    return r


def null_estimate(rule_result: Rule, d: int):
    """The null-rule estimate of one region from its rule result (or_rule's
    class sums and magnitudes).  Returns a dict of the NullOut fields."""
    q = NullOut()
    lib().or_null_estimate(C.byref(rule_result._raw), _p(null_table(d)), C.byref(q))
    return {"nul": np.array(q.nul[:]), "e": np.array(q.e[:]), "r": q.r, "est": q.est,
            "est_alt": q.est_alt, "noise": q.noise, "band": q.band, "regime": q.regime,
            "regime_tie": bool(q.regime_tie)}


def rule_regions_est(family: int, a, u, c, h, estimator=EST_NULL_RULES):
    """Rule over n regions with the chosen error estimator, as the loop uses
    it: dict of i7, err, vol, scale, err_band, err_alt, axis, axis_tie,
    split_bad."""
    c = _f64(c)
    h = _f64(h)
    n, d = c.shape
    fh = _FamilyHandle(family, a, u)
    out = {k: np.zeros(n) for k in ("i7", "err", "vol", "scale", "err_band", "err_alt")}
    ints = {k: np.zeros(n, dtype=np.int32) for k in ("axis", "axis_tie", "split_bad")}
    nw = null_table(d) if estimator == EST_NULL_RULES else None
    lib().or_rule_regions_est(C.byref(fh.s), n, _p(c), _p(h), None if nw is None else _p(nw),
                              _p(out["i7"]), _p(out["err"]), _p(out["vol"]),
                              _p(ints["axis"], C.c_int32), _p(ints["axis_tie"], C.c_int32),
                              _p(ints["split_bad"], C.c_int32), _p(out["scale"]),
                              _p(out["err_band"]), _p(out["err_alt"]))
    out.update(ints)
    return out


def rule_regions(family: int, a, u, c, h):
    """Rule over n regions (c, h: n x d arrays).  Returns a dict of arrays."""
    c = _f64(c)
    h = _f64(h)
    n, d = c.shape
    fh = _FamilyHandle(family, a, u)
    out = {k: np.zeros(n) for k in ("i7", "i5", "err", "vol", "i7abs")}
    ints = {k: np.zeros(n, dtype=np.int32) for k in ("axis", "axis_tie", "split_bad")}
    lib().or_rule_regions(C.byref(fh.s), n, _p(c), _p(h), _p(out["i7"]), _p(out["i5"]),
                          _p(out["err"]), _p(out["vol"]), _p(ints["axis"], C.c_int32),
                          _p(ints["axis_tie"], C.c_int32), _p(ints["split_bad"], C.c_int32),
                          _p(out["i7abs"]))
    out.update(ints)
    return out


def gk_nodes(d: int) -> int:
    return 15 ** d


def rule_gk(c, h, f=None, family=None, a=None, u=None):
    """Tensor-product Gauss-Kronrod rule on one region; f a Python callable
    or a built-in family.  Returns (GkOut fields as a dict, E ndarray)."""
    c = _f64(c)
    h = _f64(h)
    d = len(c)
    E = np.zeros(d)
    out = GkOut()
    L = lib()
    if f is not None:
        def cb(xp, dd, _ctx):
            return float(f(np.ctypeslib.as_array(xp, shape=(dd,)).copy()))
        cfun = INTEGRAND(cb)
        L.or_rule_gk(d, _p(c), _p(h), C.cast(cfun, C.c_void_p), None, _p(gk_table()), _p(E),
                     C.byref(out))
    else:
        fh = _FamilyHandle(family, a, u)
        fn = C.cast(L.or_family_eval, C.c_void_p)
        L.or_rule_gk(d, _p(c), _p(h), fn, C.cast(C.pointer(fh.s), C.c_void_p), _p(gk_table()),
                     _p(E), C.byref(out))
    r = {k: getattr(out, k) for k, _ in GkOut._fields_}
    for k in ("axis_tie", "flat", "split_bad"):
        r[k] = bool(r[k])
    return r, E


def rule_gk_regions(family: int, a, u, c, h):
    """Gauss-Kronrod rule over n regions (c, h: n x d).  Returns a dict of
    arrays: ik, ig, err, vol, scale, axis, axis_tie, split_bad."""
    c = _f64(c)
    h = _f64(h)
    n, d = c.shape
    fh = _FamilyHandle(family, a, u)
    out = {k: np.zeros(n) for k in ("ik", "ig", "err", "vol", "scale")}
    ints = {k: np.zeros(n, dtype=np.int32) for k in ("axis", "axis_tie", "split_bad")}
    lib().or_rule_gk_regions(C.byref(fh.s), n, _p(c), _p(h), _p(gk_table()), _p(out["ik"]),
                             _p(out["ig"]), _p(out["err"]), _p(out["vol"]),
                             _p(ints["axis"], C.c_int32), _p(ints["axis_tie"], C.c_int32),
                             _p(ints["split_bad"], C.c_int32), _p(out["scale"]))
    out.update(ints)
    return out


def pairwise_sum(v) -> float:
    v = _f64(v)
    return float(lib().or_pairwise_sum(_p(v), len(v)))


def auto_splits(d: int, cap: int) -> int:
    return int(lib().or_auto_splits(d, cap))


def partition(lo, hi, s: int):
    lo = _f64(lo)
    hi = _f64(hi)
    d = len(lo)
    n = s ** d
    c = np.zeros((n, d))
    h = np.zeros((n, d))
    lib().or_partition(d, _p(lo), _p(hi), s, _p(c), _p(h))
    return c, h


def classify(i7, err, vol, split_bad, vol_omega, budget, rel_tol=0.0, classifier=0, scale=None,
             err_band=None):
    i7, err, vol = _f64(i7), _f64(err), _f64(vol)
    sc = None if scale is None else _f64(scale)
    eb = None if err_band is None else _f64(err_band)
    sb = np.ascontiguousarray(np.asarray(split_bad, dtype=np.int32))
    n = len(i7)
    flags = np.zeros(n, dtype=np.uint8)
    ri, re_ = C.c_double(), C.c_double()
    ties = C.c_int64()
    ns = lib().or_classify_band(0, n, _p(i7), _p(err), _p(vol), _p(sb, C.c_int32),
                                None if sc is None else _p(sc), None if eb is None else _p(eb),
                                vol_omega, budget, rel_tol, classifier, _p(flags, C.c_uint8),
                                C.byref(ri), C.byref(re_), C.byref(ties))
    return dict(flags=flags, n_split=int(ns), ret_i=ri.value, ret_e=re_.value,
                near_ties=int(ties.value))


def bisect(c, h, axis, flags):
    c, h = _f64(c), _f64(h)
    n, d = c.shape
    ax = np.ascontiguousarray(np.asarray(axis, dtype=np.int32))
    fl = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    ns = int(fl.astype(bool).sum())
    co = np.zeros((2 * ns, d))
    ho = np.zeros((2 * ns, d))
    lib().or_bisect(d, n, _p(c), _p(h), _p(ax, C.c_int32), _p(fl, C.c_uint8), _p(co), _p(ho))
    return co, ho


@dataclass
class IntegrateResult:
    integral: float
    error: float
    regions_evaluated: int
    function_evals: int
    final_active: int
    iterations: int
    status: int
    near_ties: int
    trace: list


def integrate(family: int, a, u, rel_tol: float, lo=None, hi=None, abs_tol: float = 1e-16,
              max_regions: int = 100000, init_splits: int = 0, max_iters: int = 0,
              classifier: int = 0, max_trace: int = 256, rule: int = RULE_GM,
              estimator: int = EST_EMBEDDED) -> IntegrateResult:
    fh = _FamilyHandle(family, a, u)
    d = len(fh.a)
    lo = _f64(np.zeros(d) if lo is None else lo)
    hi = _f64(np.ones(d) if hi is None else hi)
    opt = _options(rel_tol, abs_tol, max_regions, init_splits, max_iters, classifier, rule,
                   estimator, d)
    res = Result()
    tr = (Trace * max_trace)()
    lib().or_integrate(C.byref(fh.s), _p(lo), _p(hi), C.byref(opt), C.byref(res), tr, max_trace)
    trace = [dict(n=t.n, n_split=t.n_split, near_ties=t.near_ties, I=t.I, E=t.E, I_ret=t.I_ret,
                  E_ret=t.E_ret, budget=t.budget) for t in tr[:min(res.iterations, max_trace)]]
    return IntegrateResult(res.integral, res.error, res.regions_evaluated, res.function_evals,
                           res.final_active, res.iterations, res.status, res.near_ties, trace)


def _lib_grad():
    L = lib()
    if not getattr(L, "_grad_sig", False):
        L.or_rule_grad.argtypes = [C.POINTER(Family), C.c_int64, _dp, _dp, _dp, _dp]
        L.or_integrate_partition.restype = C.c_int32
        L.or_integrate_partition.argtypes = [C.POINTER(Family), _dp, _dp, C.POINTER(Options),
                                             C.POINTER(Result), _dp, _dp, C.c_int64,
                                             C.POINTER(C.c_int64)]
        L._grad_sig = True
    return L


def rule_grad(family: int, a, u, c, h):
    """Frozen-partition quadrature Q and dQ/d(a, u) (2d values)."""
    c, h = _f64(c), _f64(h)
    n, d = c.shape
    fh = _FamilyHandle(family, a, u)
    g = np.zeros(2 * d)
    q = C.c_double()
    _lib_grad().or_rule_grad(C.byref(fh.s), n, _p(c), _p(h), _p(g), C.byref(q))
    return g, q.value


def integrate_partition(family: int, a, u, rel_tol: float, lo=None, hi=None,
                        abs_tol: float = 1e-16, max_regions: int = 100000, max_leaves=None,
                        init_splits: int = 0, max_iters: int = 0, classifier: int = 0,
                        estimator: int = EST_EMBEDDED):
    """or_integrate plus the final partition (leaves as n x d arrays)."""
    fh = _FamilyHandle(family, a, u)
    d = len(fh.a)
    lo = _f64(np.zeros(d) if lo is None else lo)
    hi = _f64(np.ones(d) if hi is None else hi)
    ml = max_leaves or max_regions
    co = np.zeros((ml, d))
    ho = np.zeros((ml, d))
    nl = C.c_int64()
    opt = _options(rel_tol, abs_tol, max_regions, init_splits, max_iters, classifier, RULE_GM,
                   estimator, d)
    res = Result()
    _lib_grad().or_integrate_partition(C.byref(fh.s), _p(lo), _p(hi), C.byref(opt), C.byref(res),
                                       _p(co), _p(ho), ml, C.byref(nl))
    k = int(nl.value)
    r = IntegrateResult(res.integral, res.error, res.regions_evaluated, res.function_evals,
                        res.final_active, res.iterations, res.status, res.near_ties, [])
    if k < 0:
        return r, None, None
    return r, co[:k].copy(), ho[:k].copy()
