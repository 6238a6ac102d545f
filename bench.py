"""Benchmark: Genz-Malik region-evals/s on the d = 8 seeded Genz workload.

Workload (one step): the four Genz families (oscillatory, Gaussian, corner
peak, C0) on [0,1]^8, a_j ~ U(0,1) rescaled to sum 6.0 / 3.5 / 1.85 / 2.0,
u_j ~ U(0,1), seeds 1..10, relative tolerances 1e-3 .. 1e-8, region pool up
to 2^24: 240 adaptive integrations through the C ABI, FP64.  value = regions
evaluated per second over the whole step (device time, CUDA events on the
library's stream).  e2e = the same through the public call, host wall clock,
with the parameter upload and the per-sweep status reads inside.

--impl reference times the CPU oracle (FP64, one thread) on a bounded sample
of the same workload.  Under torchrun every rank runs the same workload as
an independent replica (the method's sweep has no data-path exchange on one
GPU); value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Genz-Malik region-evals/s (d=8 Genz families, FP64)"
UNIT = "region-evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gm", choices=["gm", "reference"])
    ap.add_argument("--tols", default="1e-3,1e-4,1e-5,1e-6,1e-7,1e-8")
    ap.add_argument("--seeds", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def workload(args):
    from paper_2511_01573_gb300 import genz_inputs as G
    tols = tuple(float(t) for t in args.tols.split(","))
    return G.genz_d8_problems(seeds=range(1, args.seeds + 1), tols=tols)


CAP = 1 << 24


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index),
                                      f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        import statistics
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """CPU oracle on a bounded sample of the workload (one thread)."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    probs = workload(args)
    per_step = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    vals = []
    sample_desc = ""
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        regions = 0
        done = 0
        for p in probs:
            # bounded: the loosest tolerances first, stop when the step's
            # time budget is spent
            if time.perf_counter() - t0 > per_step:
                break
            r = O.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=min(CAP, 1 << 20))
            regions += r.regions_evaluated
            done += 1
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            vals.append(regions / dt)
            sample_desc = f"first {done} of {len(probs)} integrations in tolerance order, pool 2^20"
    v = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "genz_d8_4families_seeds1-10_tol1e-3..1e-8_cap2^24"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args, seconds):
    from oracle import oracle as O
    O.build()
    probs = workload(args)
    t0 = time.perf_counter()
    regions = 0
    done = 0
    for p in probs:
        if time.perf_counter() - t0 > seconds:
            break
        r = O.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=min(CAP, 1 << 20))
        regions += r.regions_evaluated
        done += 1
    dt = time.perf_counter() - t0
    return {"value": regions / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} of {len(probs)} integrations in tolerance order "
                      f"({dt:.1f} s, pool 2^20)"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local
    torch.cuda.set_device(dev)
    from paper_2511_01573_gb300 import gmq
    probs = workload(args)
    stream = torch.cuda.Stream(device=dev)
    ctx = gmq.Context(device=dev, stream=stream)
    ctx.profile(True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        regions = 0
        sweeps = 0
        for p in probs:
            r = ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=CAP)
            regions += r.regions_evaluated
            sweeps += r.iterations
        return regions, sweeps

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.profile_reset()
    total_ms = 0.0
    regions = sweeps = 0
    launches0 = ctx.launch_count()
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush between timed steps (outside the events)
            torch.cuda.synchronize()
            barrier()
            with torch.cuda.stream(stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rg, sw = step()
                e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            total_ms += e0.elapsed_time(e1)
            regions += rg
            sweeps += sw
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_read()
    # e2e: host wall clock through the public call
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_regions = 0
    e2e_sweeps = 0
    for _ in range(args.steps):
        rg, sw = step()
        e2e_regions += rg
        e2e_sweeps += sw
    e2e_s = time.perf_counter() - t0

    ms_step = total_ms / args.steps
    my_time = total_ms / 1000.0
    my_regions = regions
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([my_time], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        rtot = torch.tensor([float(my_regions)], dtype=torch.float64, device=dev)
        dist.all_reduce(rtot, op=dist.ReduceOp.SUM)
        my_time = float(t.item())
        my_regions = float(rtot.item())
    value = my_regions / my_time
    if rank != 0:
        return
    rule = prof["rule"]
    # FP64 roofline of the rule kernel: executed FP64 flops per region of the
    # workload's mix (measured once with ncu, see profiles/) over the rule
    # kernel's event-timed launches
    flops_per_region = float(os.environ.get("GMQ_RULE_FLOPS_PER_REGION", "0")) or None
    peak_fp64 = 2 * 2 * 152 * 2070e6 / 1e9  # GFLOP/s: 2 FP64 FMA lanes/clk/SM
    roof = None
    if rule["launches"] and flops_per_region:
        avg_s = rule["ms"] / 1000.0 / rule["launches"]
        per_launch = flops_per_region * rule["regions"] / rule["launches"]
        ach = per_launch / avg_s / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": peak_fp64, "unit": "GFLOP/s",
                "frac": ach / peak_fp64, "traffic": None}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"genz_d8_4families_seeds1-{args.seeds}_tol{args.tols}_cap2^24",
                   "integrations_per_step": len(probs), "regions_per_step": regions // args.steps,
                   "sweeps_per_step": sweeps // args.steps, "l2": "flushed between steps",
                   "parallelism": f"replicas{ws}"},
        "gpu_launches": launches,
        "kernels": prof,
        "roofline": roof,
        "e2e": {"value": e2e_regions / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": len(probs) * 4 * 8 * 8,
                "d2h_bytes_per_step": (e2e_sweeps // args.steps) * 80},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
