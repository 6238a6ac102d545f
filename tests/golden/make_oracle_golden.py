"""Writes oracle_integrations.json: the CPU oracle's results for the paper's
test functions f1..f7 (paper Sec. 4, the integrand list; f6 as read in the
paper-readings of this project: zero when any x_i exceeds (3 + i)/10) on
[0,1]^3 at relative tolerance 1e-6, and the d = 3 product-peak
configuration (a_j = 5, u_j = 1/2, tolerance 1e-6, cap 1e5).  Calls only
oracle/; each case keeps the oracle's per-sweep trace (region and split
counts, near-tie decisions, global estimates).  A regression fixture for the oracle, not a pin of it (the pins are
in tests/test_oracle_*.py).

Run from the repository root: python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2511_01573_gb300 import genz_inputs as G  # noqa: E402


def cases():
    out = []
    for k in range(1, 8):
        p = G.paper_integrand(k, 3)
        out.append((p.label + "_d3", p, 1 << 18))
    p = G.product_peak_d3()
    out.append(("product_peak_d3_a5", p, 100000))
    return out


def run(p, cap):
    r = O.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=cap)
    return {"integral": r.integral.hex(), "integral_dec": repr(r.integral),
            "error": r.error.hex(), "regions_evaluated": r.regions_evaluated,
            "function_evals": r.function_evals, "iterations": r.iterations,
            "status": r.status, "near_ties": r.near_ties,
            "trace": [{"n": t["n"], "n_split": t["n_split"], "near_ties": t["near_ties"],
                       "I": t["I"], "E": t["E"], "budget": t["budget"]} for t in r.trace]}


def main():
    rows = []
    for name, p, cap in cases():
        rows.append({"name": name, "family": p.family, "dim": p.dim, "a": list(map(float, p.a)),
                     "u": list(map(float, p.u)), "rel_tol": p.rel_tol, "max_regions": cap,
                     "result": run(p, cap)})
    with open(os.path.join(HERE, "oracle_integrations.json"), "w") as f:
        json.dump({"source": "tests/golden/make_oracle_golden.py (CPU oracle only)",
                   "cases": rows}, f, indent=1)


if __name__ == "__main__":
    main()
