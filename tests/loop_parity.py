"""End-to-end comparison of one adaptive run of the CUDA path with the
oracle's run of the same problem (paper Sec. 3 loop, Fig. 1a).

The two sides evaluate the same regions in every sweep until a decision
that rounding may legitimately flip: a classification or split-axis choice
inside the oracle's near-tie band, or a convergence test whose error sum
lies within 1e-11 of the budget.  So:

* every sweep up to and including the first flagged one evaluates the same
  number of regions, with global estimates I and E within 1e-12 of |I|;
* every sweep before it splits the same number of regions;
* when the whole run agrees anyway (same status, sweep count, per-sweep
  region and split counts), the final integral and error agree to 1e-12 of
  |I|, flags or not;
* when it does not, the divergence comes at or after a flagged sweep, and
  both runs still agree within the error both report.

No branch of this check can pass without asserting.
"""
from __future__ import annotations

STOP_BAND = 1e-11


def first_flagged_sweep(o_trace):
    """Index of the first sweep whose decisions the oracle flags (len if
    none): near-tie classification or axis decisions, or an error sum
    within STOP_BAND of the budget."""
    for i, t in enumerate(o_trace):
        if t["near_ties"] > 0:
            return i
        if abs(t["E"] - t["budget"]) <= STOP_BAND * max(abs(t["I"]), t["budget"]):
            return i
    return len(o_trace)


def assert_loop_parity(o, g, g_trace, rel=1e-12):
    """o: the oracle's IntegrateResult (with its per-sweep trace); g, g_trace:
    the CUDA path's result and gmq_last_trace records.  Returns the index of
    the first flagged sweep (len(o.trace) when none)."""
    ot = o.trace
    assert len(ot) == o.iterations, "oracle trace truncated: raise max_trace"
    k = first_flagged_sweep(ot)
    m = min(k + 1, len(ot))
    assert len(g_trace) >= m, (len(g_trace), m, k)
    scale = max(abs(o.integral), abs(g.integral))
    for i in range(m):
        a, b = g_trace[i], ot[i]
        assert a["n"] == b["n"], ("sweep", i, a["n"], b["n"])
        si = max(abs(b["I"]), scale)
        assert abs(a["I"] - b["I"]) <= rel * si + 1e-300, ("sweep", i, a["I"], b["I"])
        assert abs(a["E"] - b["E"]) <= rel * si + 1e-300, ("sweep", i, a["E"], b["E"])
        if i < k:
            assert a["n_split"] == b["n_split"], ("sweep", i, a["n_split"], b["n_split"])
    same = ((g.status, g.iterations, g.regions_evaluated) ==
            (o.status, o.iterations, o.regions_evaluated) and
            [t["n"] for t in g_trace] == [t["n"] for t in ot] and
            [t["n_split"] for t in g_trace] == [t["n_split"] for t in ot])
    if same:
        assert abs(g.integral - o.integral) <= rel * abs(o.integral) + 1e-300, (
            g.integral, o.integral)
        assert abs(g.error - o.error) <= rel * abs(o.integral) + 1e-300, (g.error, o.error)
    else:
        # a flagged decision explains the divergence (checked sweep by sweep
        # above), and the two estimates agree within what both report
        assert k < len(ot), "runs diverged without a flagged decision"
        assert abs(g.integral - o.integral) <= g.error + o.error + rel * abs(o.integral), (
            g.integral, g.error, o.integral, o.error)
    return k


def oracle_integrate_job(job):
    """One oracle integration in a worker process (spawned, so it is safe
    after CUDA has been initialised in the parent): job = (family, a, u,
    rel_tol, max_regions)."""
    from oracle import oracle as O
    fam, a, u, tol, cap = job
    return O.integrate(fam, a, u, tol, max_regions=cap)


def oracle_integrate_many(jobs, procs=None):
    """The oracle on several problems at once, one spawned process each (at
    most the host's cores); results in job order."""
    import multiprocessing as mp
    import os
    from oracle import oracle as O
    O.build()  # once, before the workers load it
    procs = max(1, min(len(jobs), procs or (os.cpu_count() or 1)))
    if procs == 1:
        return [oracle_integrate_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(oracle_integrate_job, jobs, chunksize=1)
