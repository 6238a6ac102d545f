"""Benchmark: Genz-Malik region-evals/s on the d = 8 seeded Genz workload.

Workload (one step): the four Genz families (oscillatory, Gaussian, corner
peak, C0) on [0,1]^8, a_j ~ U(0,1) rescaled to sum 6.0 / 3.5 / 1.85 / 2.0,
u_j ~ U(0,1), seeds 1..10, relative tolerances 1e-3 .. 1e-8, region pool up
to 2^24: 240 adaptive integrations through the C ABI, FP64.  value = regions
evaluated per second over the whole step (device time, CUDA events on the
library's stream).  e2e = the same through the public call, host wall clock,
with the parameter upload and the per-sweep status reads inside.

--impl reference times the CPU oracle (FP64, one process per host core) on a bounded sample
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
    ap.add_argument("--no-time-to-tol", action="store_true")
    ap.add_argument("--no-nodewise-step", action="store_true",
                    help="skip the comparison step with node-wise FP64 evaluation")
    ap.add_argument("--probe-rule", default=None,
                    help="profiling probe: family codes (e.g. 0,1,2,3,4); runs the rule "
                         "kernel 3 times per family on 2^20 random regions (--dim, default 8) "
                         "after a warm-up call, and exits")
    ap.add_argument("--probe-split", action="store_true",
                    help="profiling probe: classify + split on 2^22 random d=8 regions")
    ap.add_argument("--probe-batch", action="store_true",
                    help="profiling probe: the d=8 tol 1e-6 problems as one batch, FP64 and mixed")
    ap.add_argument("--probe-gk", default=None,
                    help="profiling probe: family codes; the Gauss-Kronrod rule kernel on 2^13 "
                         "random d=4 regions, three launches per family")
    ap.add_argument("--probe-grad", default=None,
                    help="profiling probe: family codes; the adjoint kernel on 2^18 random "
                         "d=8 regions, three calls per family")
    ap.add_argument("--eval-mode", type=int, default=0,
                    help="with --probe-rule / --probe-grad: gmq_set_eval_mode (0 separable, "
                         "1 node-wise)")
    ap.add_argument("--host-loop", action="store_true",
                    help="with --probe-batch: the host-driven sweep loop instead of the graph")
    ap.add_argument("--kernel-sweep", action="store_true",
                    help="isolated rule / classify / split rates against the region count")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="the measured FP64 and FP32 issue rates (fused multiply-add, add, "
                         "multiply chains) with the SM clocks sampled meanwhile")
    ap.add_argument("--estimators", action="store_true",
                    help="the d=8 workload with the embedded and the null-rule error estimate: "
                         "time, regions and true error against the closed forms per tolerance")
    ap.add_argument("--all-configs", action="store_true",
                    help="report the other workloads at full size (d=3; d=12 FP64 against "
                         "mixed; the 4096 batched integrals; the 1024 gradient sets)")
    ap.add_argument("--seeds-d12", type=int, default=10)
    ap.add_argument("--only", default="c1,c3,c4,c5",
                    help="--all-configs: the workloads to run (c1, c3, c4, c5)")
    ap.add_argument("--grad-sets", type=int, default=1024)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--gk", action="store_true",
                    help="with --all-configs: also the Gauss-Kronrod rule against Genz-Malik")
    ap.add_argument("--lanes", type=int, default=1)
    ap.add_argument("--dim", type=int, default=8, help="with --probe-rule: the dimension")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def workload(args):
    from paper_2511_01573_gb300 import genz_inputs as G
    tols = tuple(float(t) for t in args.tols.split(","))
    return G.genz_d8_problems(seeds=range(1, args.seeds + 1), tols=tols)


CAP = 1 << 24

# FP64 work of the rule kernel per region at d = 8 (401 nodes), per family:
# FP64 thread-instructions (sm__thread_inst_executed_pipe_fp64_pred_on) and
# flops (FMA = 2), from the ncu counters of a launch over 2^20 regions
# (bench.py --probe-rule under ncu).  The counts are fixed by the integrand,
# d and the compiled kernel: the four families take no data-dependent
# branch.  They hold for the kernel sources whose fingerprint is
# RULE_COUNTS_SHA16; when those sources change the counts must be taken
# again (tests/test_bench_counts.py fails until they are), and until then
# the roofline reports no fraction.  Family codes: 0 oscillatory, 1 product
# peak, 2 corner peak, 3 Gaussian, 4 C0.
RULE_FP64_INST_D8 = {0: 5631.0, 1: 2476.0, 2: 4829.0, 3: 4136.0, 4: 4080.0}
RULE_FP64_FLOPS_D8 = {0: 8882.0, 1: 3778.0, 2: 6075.0, 3: 6184.0, 4: 6128.0}
RULE_COUNTS_SOURCES = ("gm_rule.cuh", "gm_region64.cuh", "gmq_families.cuh",
                       "gm_math_tables.cuh", "gmq_common.cuh")
RULE_COUNTS_SHA16 = "fcb577d59be93b60"


# FP32 work of the mixed rule kernel (k_rule_mixed_reg, one thread per
# region) per region at d = 12 (4409 nodes), corner peak and Gaussian (the
# d = 12 mixed workload): FP32 lane operations, i.e. FP32 thread
# instructions with each paired instruction (FADD2 / FMUL2 / FFMA2) counted
# twice (sm__sass_thread_inst_executed_op_fp32_pred_on +
# sm__sass_thread_inst_executed_ops_fadd2_fmul2_ffma2_pred_on, ncu, 2^20
# regions; bench.py --probe-rule 2,3 --precision 1 --dim 12).  Tied to the
# mixed kernel's sources as the FP64 counts are to the FP64 kernel's.
MIXED_FP32_OPS_D12 = {2: 116237.0, 3: 134179.0}
MIXED_COUNTS_SOURCES = ("gm_rule_mixed.cuh", "gm_region32.cuh", "gm_region64.cuh",
                        "gmq_families.cuh", "gm_math_tables.cuh", "gmq_common.cuh")
MIXED_COUNTS_SHA16 = "c1f3307de3c65ba1"


def rule_source_fingerprint(files=RULE_COUNTS_SOURCES):
    """First 16 hex digits of the SHA-256 of a rule kernel's sources (file
    name, then contents, in the order given; the FP64 kernel's by default)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2511_01573_gb300", "csrc")
    for f in files:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


RULE_DRAM_BYTES_PER_REGION_D8 = 142.8


def mixed_roofline(ctx, stream, probe32):
    """Roofline of the mixed rule kernel on the d = 12 mixed workload's
    families (corner peak, Gaussian): one thread per region (the register
    walk) over 2^20 random sub-boxes of [0,1]^12, one warm-up call and three
    event-timed launches per family on the context stream; achieved FP32
    lane operations per second (MIXED_FP32_OPS_D12 per region) against the
    measured FP32 issue rate probe32 (lane operations per second)."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    n, d = 1 << 20, 12
    g = torch.Generator(device="cuda").manual_seed(12)
    lo = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.9
    w = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.05 + 1e-3
    c = (lo + 0.5 * w).contiguous()
    h = (0.5 * w).contiguous()
    ops = secs = 0.0
    per = {}
    for fam in sorted(MIXED_FP32_OPS_D12):
        a, u = G.seed_genz(1, fam, d, G.GENZ_TARGET_SUM[fam])
        ctx.eval_rule(fam, a, u, c[:, :256].contiguous(), h[:, :256].contiguous(), lanes=1,
                      precision=gmq.MIXED)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(3):
                ctx.eval_rule(fam, a, u, c, h, lanes=1, precision=gmq.MIXED)
            e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1000.0
        per[G.FAMILY_NAMES[fam]] = {"ms_per_launch": t / 3 * 1000.0, "regions_per_s": 3 * n / t,
                                    "G_fp32_lane_ops_per_s": 3 * n * MIXED_FP32_OPS_D12[fam] / t / 1e9}
        ops += 3 * n * MIXED_FP32_OPS_D12[fam]
        secs += t
    del c, h, lo, w
    current = rule_source_fingerprint(MIXED_COUNTS_SOURCES) == MIXED_COUNTS_SHA16
    ach = ops / secs / 1e9
    peak = probe32 / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G FP32 lane-ops/s",
            "frac": ach / peak if current else None, "traffic": None,
            "kernel": "k_rule_mixed_reg<FAM, 12> (mixed-precision rule evaluation, d = 12)",
            "workload": "2^20 random sub-boxes of [0,1]^12, corner peak and Gaussian, "
                        "three launches each, kernel timed alone",
            "peak_basis": "measured: FP32 fused multiply-add chains of the issue-rate probe "
                          "(gmq_probe_fp_rate) in this run",
            "counts_match_source": current, "fp32_lane_ops_per_region": {
                G.FAMILY_NAMES[f]: v for f, v in MIXED_FP32_OPS_D12.items()},
            "by_family": per}


def eval_modes(ctx, stream):
    """The FP64 rule kernel's two ways of evaluating f at the nodes
    (gmq_set_eval_mode) on the benchmark's families at d = 8: one thread per
    region over 2^20 random sub-boxes of [0,1]^8, one warm-up call and three
    event-timed launches per family and mode on the context stream.  The
    default forms each node's S from per-axis terms (separable); node-wise
    evaluates f from every node's coordinates, as an integrand without that
    form would be.  Both evaluate g at every node."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    n, d = 1 << 20, 8
    g = torch.Generator(device="cuda").manual_seed(8)
    lo = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.9
    w = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.05 + 1e-3
    c = (lo + 0.5 * w).contiguous()
    h = (0.5 * w).contiguous()
    out = {}
    for name, mode in (("separable", gmq.EVAL_SEPARABLE), ("nodewise", gmq.EVAL_NODEWISE)):
        ctx.set_eval_mode(mode)
        per = {}
        for fam in G.GENZ_D8_FAMILIES:
            a, u = G.seed_genz(1, fam, d, G.GENZ_TARGET_SUM[fam])
            ctx.eval_rule(fam, a, u, c[:, :256].contiguous(), h[:, :256].contiguous(), lanes=1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for _ in range(3):
                    ctx.eval_rule(fam, a, u, c, h, lanes=1)
                e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1000.0
            per[G.FAMILY_NAMES[fam]] = {"ms_per_launch": t / 3 * 1000.0, "regions_per_s": 3 * n / t}
        out[name] = per
    ctx.set_eval_mode(gmq.EVAL_SEPARABLE)
    out["separable_over_nodewise"] = {
        f: out["nodewise"][f]["ms_per_launch"] / out["separable"][f]["ms_per_launch"]
        for f in out["separable"]}
    out["workload"] = "2^20 random sub-boxes of [0,1]^8, one thread per region, kernel timed alone"
    del c, h, lo, w
    return out


def time_to_tol(ctx, stream, tol):
    """Wall time (CUDA events) for the 40 d = 8 problems at one tolerance,
    FP64 against the mixed form, and the mixed results' largest relative
    difference from the FP64 results."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    probs = G.genz_d8_problems(tols=(tol,))
    out = {"tol": tol, "problems": len(probs)}
    vals = {}
    for name, prec in (("fp64", gmq.FP64), ("mixed", gmq.MIXED)):
        for p in probs[:4]:
            ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=CAP, precision=prec)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=CAP, precision=prec)
               for p in probs]
        e1.record(stream)
        torch.cuda.synchronize()
        vals[name] = res
        out[f"{name}_s"] = e0.elapsed_time(e1) / 1000.0
        out[f"{name}_regions"] = sum(r.regions_evaluated for r in res)
        out[f"{name}_converged"] = sum(1 for r in res if r.status == 0)
    out["speedup_mixed_over_fp64"] = out["fp64_s"] / out["mixed_s"]
    out["mixed_max_rel_diff_vs_fp64"] = max(
        abs(m.integral - f.integral) / abs(f.integral) for m, f in zip(vals["mixed"], vals["fp64"]))
    # batched form (FP64, one graph launch for all 40 problems)
    ctx.integrate_batch(probs[:4], max_regions=CAP)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = ctx.integrate_batch(probs, max_regions=CAP, pool_regions=1 << 26)
    e1.record(stream)
    torch.cuda.synchronize()
    out["batched_s"] = e0.elapsed_time(e1) / 1000.0
    out["batched_regions"] = sum(r.regions_evaluated for r in res)
    out["batched_converged"] = sum(1 for r in res if r.status == 0)
    out["speedup_batched_over_fp64"] = out["fp64_s"] / out["batched_s"]
    out["batched_max_rel_diff_vs_fp64"] = max(
        abs(b.integral - f.integral) / abs(f.integral) for b, f in zip(res, vals["fp64"]))
    # batched mixed form (one graph launch, FP32 integrand)
    ctx.integrate_batch(probs[:4], max_regions=CAP, precision=gmq.MIXED)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = ctx.integrate_batch(probs, max_regions=CAP, pool_regions=1 << 26, precision=gmq.MIXED)
    e1.record(stream)
    torch.cuda.synchronize()
    out["batched_mixed_s"] = e0.elapsed_time(e1) / 1000.0
    out["batched_mixed_regions"] = sum(r.regions_evaluated for r in res)
    out["batched_mixed_converged"] = sum(1 for r in res if r.status == 0)
    out["speedup_batched_mixed_over_fp64"] = out["fp64_s"] / out["batched_mixed_s"]
    out["speedup_batched_mixed_over_mixed"] = out["mixed_s"] / out["batched_mixed_s"]
    out["batched_mixed_max_rel_diff_vs_fp64"] = max(
        abs(b.integral - f.integral) / abs(f.integral) for b, f in zip(res, vals["fp64"]))
    return out


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


def aggregate_over_ranks(my_time_s, my_regions, world_size, device="cpu"):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the regions of all ranks (no data-path collective; only these two
    numbers cross ranks, after the timed region)."""
    if world_size <= 1:
        return float(my_time_s), float(my_regions)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(my_time_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    r = torch.tensor([float(my_regions)], dtype=torch.float64, device=device)
    dist.all_reduce(r, op=dist.ReduceOp.SUM)
    return float(t.item()), float(r.item())


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _oracle_one(job):
    """One integration by the CPU oracle in a host process, unless the
    sample's wall-clock deadline has passed.  Returns (regions, done,
    integral, status)."""
    p, deadline, cap = job
    if time.time() > deadline:
        return 0, 0, 0.0, -1
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    r = O.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=cap)
    return r.regions_evaluated, 1, r.integral, r.status


def _oracle_load(_):
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    O.lib()
    return 0


ORACLE_CAP = 1 << 16  # bounds one integration to about a second of oracle time


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The unchanged single-threaded oracle, one process per host core
    (spawned, so it is safe after CUDA is initialised).  A sample hands the
    problems out in tolerance order to whichever process is free; problems
    not started by the deadline are skipped."""

    def __init__(self, procs):
        import multiprocessing as mp
        from oracle import oracle as O
        O.build()  # once, before the workers load it
        self.procs = procs
        self.pool = None
        if procs > 1:
            self.pool = mp.get_context("spawn").Pool(procs)
            self.pool.map(_oracle_load, range(procs), chunksize=1)

    def run(self, probs, seconds, cap=None):
        t0 = time.perf_counter()
        jobs = [(p, time.time() + seconds, cap or ORACLE_CAP) for p in probs]
        if self.pool:
            outs = self.pool.map(_oracle_one, jobs, chunksize=1)
        else:
            outs = [_oracle_one(j) for j in jobs]
        wall = time.perf_counter() - t0
        self.last = outs
        return sum(o[0] for o in outs) / wall, sum(o[1] for o in outs), wall

    def close(self):
        if self.pool:
            self.pool.close()
            self.pool.join()


def run_reference(args):
    """CPU oracle on a bounded sample of the workload, all host cores."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    probs = workload(args)
    cores = host_cores()
    pool = OraclePool(cores)
    per_step = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    vals, walls = [], []
    sample_desc = ""
    for step in range(args.warmup + args.steps):
        v, done, wall = pool.run(probs, per_step)
        if step >= args.warmup:
            vals.append(v)
            walls.append(wall)
            sample_desc = (f"{done} of {len(probs)} integrations in tolerance order, "
                           f"{cores} processes, problems started within {per_step:.1f} s "
                           f"({wall:.1f} s), pool 2^16")
    pool.close()
    v = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(walls) / len(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"genz_d8_4families_seeds1-{args.seeds}_tol{args.tols}_cap2^24",
                       "integrations_per_step": len(probs), "parallelism": "replicas1",
                       "sample": "each step a bounded sample of the integrations"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args, seconds):
    """The oracle on one core and on all host cores, each on a bounded
    sample of the workload (the loosest tolerances first)."""
    probs = workload(args)
    one = OraclePool(1)
    v1, done1, wall1 = one.run(probs, seconds)
    cores = host_cores()
    pool = OraclePool(cores)
    v, done, wall = pool.run(probs, seconds)
    pool.close()
    # time to 1e-6 on the 40 tolerance-1e-6 problems, all cores, pool 2^22
    from paper_2511_01573_gb300 import genz_inputs as G
    p6 = G.genz_d8_problems(tols=(1e-6,))
    pool = OraclePool(cores)
    _, done6, wall6 = pool.run(p6, 3600.0, cap=1 << 22)
    conv6 = sum(1 for o in pool.last if o[3] == 0)
    pool.close()
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} of {len(probs)} integrations in tolerance order, one process "
                      f"per core, started within {seconds:.0f} s ({wall:.1f} s), pool 2^16",
            "single_core": {"value": v1, "cores": 1,
                            "sample": f"first {done1} integrations ({wall1:.1f} s)"},
            "time_to_1e-6": {"s": wall6, "problems": done6, "converged": conv6,
                             "cores": cores, "pool": "2^22 per integration"}}


def probe_rule(args):
    """The rule kernel alone on 2^20 random sub-boxes of [0,1]^d (d = --dim,
    default 8: about 150 MB of inputs and outputs, more than L2), one
    warm-up call then three launches per family, for ncu captures; prints
    the event-timed rate."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    n, d = 1 << 20, args.dim
    g = torch.Generator(device="cuda").manual_seed(1)
    lo = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.9
    w = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.05 + 1e-3
    c = (lo + 0.5 * w).contiguous()
    h = (0.5 * w).contiguous()
    ctx = gmq.Context(0)
    ctx.set_eval_mode(args.eval_mode)
    ctx.profile(True)
    for fam in (int(x) for x in args.probe_rule.split(",")):
        a, u = G.seed_genz(1, fam, d, G.GENZ_TARGET_SUM.get(fam, 2.0))
        # warm-up on a few regions (loads the kernel's module) before the timed launches
        ctx.eval_rule(fam, a, u, c[:, :256].contiguous(), h[:, :256].contiguous(),
                      lanes=args.lanes, precision=args.precision)
        ctx.profile_reset()
        for _ in range(3):
            ctx.eval_rule(fam, a, u, c, h, lanes=args.lanes, precision=args.precision)
        p = ctx.profile_read()["rule"]
        print(f"family {fam} lanes {args.lanes} precision {args.precision}: {p['launches']} "
              f"launches, {p['ms'] / p['launches']:.3f} ms/launch, "
              f"{n * p['launches'] / p['ms'] * 1e3:.4g} regions/s", flush=True)
    ctx.close()


def probe_grad(args):
    """The adjoint kernel (k_rule_grad_sep, or k_rule_grad with --eval-mode 1)
    alone on 2^18 random sub-boxes of [0,1]^8 (17 output rows,
    about 70 MB of inputs and outputs), three calls per family, for ncu
    captures; prints the event-timed rate of the kernel and of the row sums."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    n, d = 1 << 18, 8
    g = torch.Generator(device="cuda").manual_seed(3)
    lo = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.9
    w = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.05 + 1e-3
    c = (lo + 0.5 * w).contiguous()
    h = (0.5 * w).contiguous()
    ctx = gmq.Context(0)
    ctx.set_eval_mode(args.eval_mode)
    ctx.profile(True)
    for fam in (int(x) for x in args.probe_grad.split(",")):
        a, u = G.seed_genz(1, fam, d, G.GENZ_TARGET_SUM.get(fam, 2.0))
        ctx.profile_reset()
        for _ in range(3):
            ctx.rule_grad(fam, a, u, c, h)
        p = ctx.profile_read()
        r, s = p["rule"], p["sum"]
        print(f"grad family {fam} d {d}: {r['launches']} launches, "
              f"{r['ms'] / r['launches']:.3f} ms/launch, "
              f"{n * r['launches'] / r['ms'] * 1e3:.4g} regions/s; row sums "
              f"{s['ms'] / max(s['launches'], 1):.3f} ms/launch", flush=True)
    ctx.close()


def probe_split(args):
    """Classify + split alone on 2^22 random d = 8 regions (three calls):
    HBM-bound kernels.  The budget is the median per-region threshold, so
    about half the regions split."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    n, d = 1 << 22, 8
    g = torch.Generator(device="cuda").manual_seed(2)
    lo = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.9
    w = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.05 + 1e-3
    c = (lo + 0.5 * w).contiguous()
    h = (0.5 * w).contiguous()
    ctx = gmq.Context(0)
    a, u = G.seed_genz(1, G.GAUSSIAN, d, 3.5)
    i7, err, vf, ax = ctx.eval_rule(G.GAUSSIAN, a, u, c, h, precision=gmq.MIXED)
    budget = float(torch.median(err / vf).item())
    ctx.profile(True)
    for _ in range(3):
        out = ctx.classify_split(c, h, i7, err, vf, ax, budget)
    p = ctx.profile_read()
    ns = out["n_split"]
    for k in ("classify", "split"):
        ms = p[k]["ms"] / p[k]["launches"]
        alg = 26.0 * n if k == "classify" else (1.0 * n + ns * (16 * d + 32 * d))
        print(f"{k}: {ms:.3f} ms/launch, n={n}, n_split={ns}, algorithmic {alg / 1e6:.1f} MB, "
              f"{alg / ms / 1e6:.1f} GB/s", flush=True)
    ctx.close()


def kernel_sweep(args):
    """Isolated kernel rates against the region count: the rule kernel over
    n = 2^16 .. 2^24 random sub-boxes of [0,1]^d for d = 3, 8, 12 (Gaussian
    family, FP64 and mixed, lanes per region chosen by the library; sizes
    whose launch would take more than about a second are skipped), and
    classify + split over n = 2^20 .. 2^24 at d = 8 with about half the
    regions split.  Event-timed, three launches each after one warm-up.
    Prints one JSON object."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    ctx = gmq.Context(0)
    ctx.profile(True)
    g = torch.Generator(device="cuda").manual_seed(3)

    def boxes(d, n):
        lo = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.9
        w = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.05 + 1e-3
        return (lo + 0.5 * w).contiguous(), (0.5 * w).contiguous()

    rows = []
    for d in (3, 8, 12):
        a, u = G.seed_genz(1, G.GAUSSIAN, d, 3.5)
        for prec in (gmq.FP64, gmq.MIXED):
            rate = None
            for lg in range(16, 25, 2):
                n = 1 << lg
                if rate is not None and n / rate > 1.0:
                    rows.append({"kernel": "rule", "d": d, "precision": prec, "n": n,
                                 "skipped": "launch over 1 s"})
                    continue
                c, h = boxes(d, n)
                ctx.eval_rule(G.GAUSSIAN, a, u, c, h, precision=prec)
                ctx.profile_reset()
                for _ in range(3):
                    ctx.eval_rule(G.GAUSSIAN, a, u, c, h, precision=prec)
                p = ctx.profile_read()["rule"]
                ms = p["ms"] / p["launches"]
                rate = n / ms * 1e3
                rows.append({"kernel": "rule", "d": d, "precision": prec, "n": n,
                             "ms": ms, "regions_per_s": rate,
                             "node_evals_per_s": rate * ((1 << d) + 2 * d * d + 2 * d + 1)})
                del c, h
    d = 8
    a, u = G.seed_genz(1, G.GAUSSIAN, d, 3.5)
    for lg in range(20, 25, 2):
        n = 1 << lg
        c, h = boxes(d, n)
        i7, err, vf, ax = ctx.eval_rule(G.GAUSSIAN, a, u, c, h, precision=gmq.MIXED)
        budget = float(torch.median(err / vf).item())
        ctx.classify_split(c, h, i7, err, vf, ax, budget)
        ctx.profile_reset()
        for _ in range(3):
            out = ctx.classify_split(c, h, i7, err, vf, ax, budget)
        p = ctx.profile_read()
        ns = out["n_split"]
        for k in ("classify", "split"):
            ms = p[k]["ms"] / p[k]["launches"]
            alg = 26.0 * n if k == "classify" else (1.0 * n + ns * (16 * d + 32 * d))
            rows.append({"kernel": k, "d": d, "n": n, "n_split": ns, "ms": ms,
                         "algorithmic_MB": alg / 1e6, "GB_per_s": alg / ms / 1e6})
        del c, h, i7, err, vf, ax, out
    print(json.dumps({"kernel_sweep": rows}), flush=True)
    ctx.close()


def probe_batch(args):
    """The 40 d = 8 problems at tolerance 1e-6 as one batch, FP64 then
    mixed (one call each after a warm-up call), for ncu launch lists of the
    batched form (--host-loop launches every sweep's kernels from the host,
    where a profiler sees them one by one); prints the event-timed seconds."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    probs = G.genz_d8_problems(tols=(1e-6,))
    stream = torch.cuda.Stream(device=0)
    ctx = gmq.Context(0, stream=stream)
    for name, prec in (("fp64", gmq.FP64), ("mixed", gmq.MIXED)):
        ctx.integrate_batch(probs[:4], max_regions=CAP, precision=prec)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = ctx.integrate_batch(probs, max_regions=CAP, pool_regions=1 << 26, precision=prec,
                                  host_loop=args.host_loop)
        e1.record(stream)
        torch.cuda.synchronize()
        info = ctx.last_batch_info()
        print(f"batch {name}: {e0.elapsed_time(e1) / 1e3:.4f} s, "
              f"{sum(r.regions_evaluated for r in res)} regions, {info['sweeps']} sweeps, "
              f"lane sweeps {info['lane_sweeps']}", flush=True)
    ctx.close()


def probe_gk(args):
    """The Gauss-Kronrod rule kernel alone on 2^13 random sub-boxes of
    [0,1]^4 (15^4 nodes each), three launches per family, for ncu captures;
    prints the event-timed rate."""
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    n, d = 1 << 13, 4
    g = torch.Generator(device="cuda").manual_seed(5)
    lo = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.9
    w = torch.rand((d, n), dtype=torch.float64, device="cuda", generator=g) * 0.05 + 1e-3
    c = (lo + 0.5 * w).contiguous()
    h = (0.5 * w).contiguous()
    ctx = gmq.Context(0)
    ctx.profile(True)
    for fam in (int(x) for x in args.probe_gk.split(",")):
        a, u = G.seed_genz(1, fam, d, G.GENZ_TARGET_SUM.get(fam, 2.0))
        ctx.profile_reset()
        for _ in range(3):
            ctx.eval_rule_gk(fam, a, u, c, h)
        p = ctx.profile_read()["rule"]
        ms = p["ms"] / p["launches"]
        print(f"gk family {fam} d {d}: {ms:.3f} ms/launch, {n / ms * 1e3:.4g} regions/s, "
              f"{n * 15 ** d / ms * 1e3:.4g} node-evals/s", flush=True)
    ctx.close()


def _closed(fam, a, u):
    """Closed forms on [0,1]^d: Gaussian erf product, oscillatory
    Re[e^{i 2 pi u1} prod (e^{i a} - 1) / (i a)], C0 exp product."""
    import cmath
    import math
    from paper_2511_01573_gb300 import genz_inputs as G
    if fam == G.GAUSSIAN:
        return _closed_gauss(a, u)[0]
    if fam == G.C0:
        return math.prod((2.0 - math.exp(-ai * ui) - math.exp(-ai * (1.0 - ui))) / ai
                         for ai, ui in zip(a, u))
    if fam == G.OSCILLATORY:
        z = cmath.exp(2j * math.pi * u[0])
        for ai in a:
            z *= (cmath.exp(1j * ai) - 1.0) / (1j * ai)
        return z.real
    if fam == G.CORNER_PEAK:
        # (1 / (d! prod a)) sum_{S} (-1)^|S| / (1 + sum_{j in S} a_j), in exact
        # rational arithmetic (the alternating sum cancels badly in FP64)
        from fractions import Fraction
        from itertools import combinations
        fa = [Fraction(x) for x in a]
        tot = Fraction(0)
        for k in range(len(fa) + 1):
            for S in combinations(fa, k):
                tot += Fraction((-1) ** k) / (1 + sum(S, Fraction(0)))
        den = Fraction(math.factorial(len(fa)))
        for x in fa:
            den *= x
        return float(tot / den)
    raise ValueError(fam)


def _closed_gauss(a, u):
    import math
    g = [math.sqrt(math.pi) / (2 * ai) * (math.erf(ai * (1 - ui)) + math.erf(ai * ui))
         for ai, ui in zip(a, u)]
    dga = [-gi / ai + ((1 - ui) * math.exp(-(ai * (1 - ui)) ** 2)
                       + ui * math.exp(-(ai * ui) ** 2)) / ai for gi, ai, ui in zip(g, a, u)]
    dgu = [math.exp(-(ai * ui) ** 2) - math.exp(-(ai * (1 - ui)) ** 2) for ai, ui in zip(a, u)]
    I = math.prod(g)
    return I, [I / gi * x for gi, x in zip(g, dga)] + [I / gi * x for gi, x in zip(g, dgu)]


def all_configs(args):
    """The other workloads beside the benchmark's own, at their full sizes:
    d = 3 product peak; d = 12 corner peak and Gaussian, FP64 against mixed
    per tolerance with both errors against the closed forms; the 4096
    batched integrals (FP64 and mixed, batched against one call per
    integral, every result against its closed form); the 1024 d = 6
    Gaussian gradient sets against the closed-form gradients; optionally the
    Gauss-Kronrod rule against Genz-Malik.  GPU times from CUDA events.
    Prints one JSON object per workload and a final summary object (a
    report, not the metric)."""
    import math
    import statistics
    import torch
    from paper_2511_01573_gb300 import autograd as AG
    from paper_2511_01573_gb300 import genz_inputs as G
    from paper_2511_01573_gb300 import gmq
    stream = torch.cuda.Stream(device=0)
    ctx = gmq.Context(0, stream=stream)

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1000.0

    def emit(key, val):
        rep[key] = val
        print(json.dumps({key: val}), flush=True)

    rep = {}
    only = set(args.only.split(","))
    if "c1" in only:
        # C1: product peak on [0,1]^3, a = 5, u = 1/2, tol 1e-6, cap 1e5
        p = G.product_peak_d3()
        ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=100000)
        r, t = timed(lambda: ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=100000))
        ex = (10 * math.atan(2.5)) ** 3
        emit("product_peak_d3", {"s": t, "regions": r.regions_evaluated, "sweeps": r.iterations,
                                 "status": r.status, "error_estimate": r.error,
                                 "rel_err_vs_closed_form": abs(r.integral - ex) / ex})
    if "c3" in only:
        # C3: d = 12 corner peak and Gaussian, FP64 against the mixed form
        rows = []
        for tol in (1e-4, 1e-5, 1e-6, 1e-7):
            for fam in (G.CORNER_PEAK, G.GAUSSIAN):
                for sd in range(1, args.seeds_d12 + 1):
                    a, u = G.seed_genz(sd, fam, 12, G.GENZ_TARGET_SUM[fam])
                    ex = _closed(fam, a, u)
                    r64, t64 = timed(lambda: ctx.integrate(fam, a, u, tol, max_regions=1 << 22))
                    rmx, tmx = timed(lambda: ctx.integrate(fam, a, u, tol, max_regions=1 << 22,
                                                           precision=gmq.MIXED))
                    rows.append({"family": G.FAMILY_NAMES[fam], "seed": sd, "tol": tol,
                                 "fp64_s": t64, "mixed_s": tmx, "fp64_regions": r64.regions_evaluated,
                                 "mixed_regions": rmx.regions_evaluated, "fp64_status": r64.status,
                                 "mixed_status": rmx.status,
                                 "fp64_rel_err": abs(r64.integral - ex) / abs(ex),
                                 "mixed_rel_err": abs(rmx.integral - ex) / abs(ex),
                                 "mixed_rel_diff_vs_fp64": abs(rmx.integral - r64.integral)
                                 / abs(r64.integral)})
        emit("d12_fp64_vs_mixed", rows)
    if "c4" in only:
        # C4: the 4096 batched integrals, FP64 and mixed, batched and one by one
        probs = G.batched_problems(count=4096)[: args.batch_count]
        bcap = 1 << 22  # per problem
        exact = [_closed(q.family, q.a, q.u) for q in probs]

        def errs(res):
            rel = [abs(x.integral - e) / abs(e) / q.rel_tol
                   for x, e, q in zip(res, exact, probs) if x.status == 0]
            fam = {}
            for x, e, q in zip(res, exact, probs):
                if x.status == 0:
                    v = abs(x.integral - e) / abs(e) / q.rel_tol
                    c = fam.setdefault(G.FAMILY_NAMES[q.family], [0, 0, 0.0])
                    c[0] += 1
                    c[1] += int(v <= 1.0)
                    c[2] = max(c[2], float(v))
            return {"converged": len(rel), "within_tol": sum(1 for v in rel if v <= 1.0),
                    "max_err_over_tol": max(rel) if rel else None,
                    "median_err_over_tol": statistics.median(rel) if rel else None,
                    "by_family_converged_within_max": fam}

        out = {"problems": len(probs)}
        for name, prec in (("fp64", gmq.FP64), ("mixed", gmq.MIXED)):
            ctx.integrate_batch(probs[:16], max_regions=bcap, precision=prec)
            res, tb = timed(lambda: ctx.integrate_batch(probs, max_regions=bcap, pool_regions=1 << 27,
                                                        precision=prec))
            info = ctx.last_batch_info()
            # one call per integral; the mixed batch runs one lane per region, so
            # the single mixed calls that it reproduces bit for bit do too
            lanes = 1 if prec == gmq.MIXED else 0
            seq, ts = timed(lambda: [ctx.integrate(q.family, q.a, q.u, q.rel_tol, max_regions=bcap,
                                                   precision=prec, lanes=lanes) for q in probs])
            st = {}
            for x in res:
                st[str(x.status)] = st.get(str(x.status), 0) + 1
            out[name] = {"batched_s": tb, "sequential_s": ts, "speedup": ts / tb,
                         "regions": sum(x.regions_evaluated for x in res), "statuses": st,
                         "identical_to_single_runs": sum(
                             1 for a, b in zip(seq, res)
                             if a.integral == b.integral and a.regions_evaluated == b.regions_evaluated),
                         "vs_closed_form": errs(res),
                         "info": {k: info[k] for k in ("sweeps", "lane_sweeps", "rule_grid", "pauses",
                                                       "evictions", "lanes_t1", "lanes_t4",
                                                       "lanes_t32", "rule_regions",
                                                       "carried_regions", "list_regions")}}
            if name == "fp64":
                fp64_res, fp64_seq_s = res, ts
        out["mixed"]["speedup_vs_fp64_sequential"] = fp64_seq_s / out["mixed"]["batched_s"]
        out["mixed"]["max_rel_diff_vs_fp64"] = max(
            abs(m.integral - f.integral) / abs(f.integral) for m, f in zip(res, fp64_res)
            if f.integral != 0.0)
        emit("batch", out)
    if "c5" in only:
        # C5: gradients of the d = 6 Gaussian over frozen partitions, tol 1e-8
        sets = G.gaussian_grad_sets(count=1024, dim=6)[: args.grad_sets]
        errs_g, errs_i, tf, tg, t_retry = [], [], 0.0, 0.0, 0.0
        caps = (1 << 24, 1 << 26, 1 << 28)
        needed = {c: 0 for c in caps}
        for a, u in sets:
            at = torch.tensor(a, requires_grad=True)
            ut = torch.tensor(u, requires_grad=True)
            # the final partition (retired leaves plus the last list) must fit in
            # max_regions: sets that outgrow it run again with four times the room
            for cap in caps:
                w0 = time.perf_counter()
                try:
                    I, t1 = timed(lambda: AG.integral(at, ut, rel_tol=1e-8, context=ctx,
                                                      max_regions=cap))
                    break
                except RuntimeError:
                    torch.cuda.synchronize()
                    t_retry += time.perf_counter() - w0
                    if cap == caps[-1]:
                        raise
            needed[cap] += 1
            _, t2 = timed(lambda: I.backward())
            tf += t1
            tg += t2
            Iex, gex = _closed_gauss(a, u)
            g = list(at.grad.numpy()) + list(ut.grad.numpy())
            errs_g.append(max(abs(x - y) for x, y in zip(g, gex)) / max(abs(y) for y in gex))
            errs_i.append(abs(float(I.detach()) - Iex) / abs(Iex))
        emit("gaussian_d6_gradients", {
            "sets": len(sets), "forward_s": tf, "adjoint_s": tg,
            "attempts_without_room_s": t_retry,
            "sets_by_partition_room": {f"2^{c.bit_length() - 1}": k for c, k in needed.items()},
            "max_rel_grad_err_vs_closed_form": max(errs_g),
            "median_rel_grad_err_vs_closed_form": statistics.median(errs_g),
            "max_rel_integral_err_vs_closed_form": max(errs_i)})
    if args.gk:
        # the tensor-product Gauss-Kronrod rule against Genz-Malik, d = 2..6
        gk_rows = []
        for fam in (G.GAUSSIAN, G.OSCILLATORY, G.C0):
            for d in (2, 3, 4, 5, 6):
                a, u = G.seed_genz(1, fam, d, G.GENZ_TARGET_SUM[fam])
                for tol in ((1e-6, 1e-9) if d <= 4 else (1e-6,)):
                    row = {"family": G.FAMILY_NAMES[fam], "d": d, "tol": tol}
                    for name, rule, cap in (("gm", gmq.RULE_GENZ_MALIK, 1 << 22),
                                            ("gk", gmq.RULE_GAUSS_KRONROD, 1 << 18)):
                        r, t = timed(lambda: ctx.integrate(fam, a, u, tol, max_regions=cap,
                                                           rule=rule))
                        row[name] = {"s": t, "regions": r.regions_evaluated,
                                     "function_evals": r.function_evals, "status": r.status,
                                     "integral": r.integral}
                    ref = _closed(fam, a, u)
                    for name in ("gm", "gk"):
                        row[name]["rel_err_vs_closed_form"] = (
                            abs(row[name]["integral"] - ref) / abs(ref))
                    gk_rows.append(row)
        emit("gauss_kronrod_vs_genz_malik", gk_rows)
    print(json.dumps({"all_configs": rep}), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.probe_peaks:
        return probe_peaks(args)
    if args.estimators:
        return estimators(args)
    if args.all_configs:
        return all_configs(args)
    if args.probe_rule:
        return probe_rule(args)
    if args.probe_split:
        return probe_split(args)
    if args.kernel_sweep:
        return kernel_sweep(args)
    if args.probe_batch:
        return probe_batch(args)
    if args.probe_gk:
        return probe_gk(args)
    if args.probe_grad:
        return probe_grad(args)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    from paper_2511_01573_gb300 import genz_inputs as G
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

    fam_regions = {}

    def step():
        regions = 0
        sweeps = 0
        for p in probs:
            r = ctx.integrate(p.family, p.a, p.u, p.rel_tol, max_regions=CAP)
            regions += r.regions_evaluated
            sweeps += r.iterations
            fam_regions[p.family] = fam_regions.get(p.family, 0) + r.regions_evaluated
        return regions, sweeps

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.profile_reset()
    fam_regions.clear()
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
    timed_fam_regions = dict(fam_regions)
    # measured FP64 issue rate of this GPU (the roofline's peak): the probe
    # kernel's fused multiply-add, add and multiply chains after a warm-up
    # launch, clocks sampled meanwhile; the pipe's peak is the fastest
    with ClockSampler(dev) as pclk:
        ctx.probe_fp_rate(gmq.FP64, iters=2000)
        probe_ops = {op: max(ctx.probe_fp_rate(gmq.FP64, op)[0] for _ in range(2))
                     for op in ctx.PROBE_OPS}
        probe32 = max(ctx.probe_fp_rate(gmq.MIXED, "fma")[0] for _ in range(2))
    probe_clocks = pclk.summary()
    probe64 = max(probe_ops.values())
    roof_mixed = mixed_roofline(ctx, stream, probe32)
    modes = eval_modes(ctx, stream)
    # e2e: host wall clock through the public call (one step), with the
    # per-launch timing events off; its device time (events around the whole
    # step) against the timed steps' shows what those events cost
    ctx.profile(False)
    flush.fill_(1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    e2e_regions, e2e_sweeps = step()
    e1.record(stream)
    e2e_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    unprofiled_ms = e0.elapsed_time(e1)
    # the same step with the FP64 rule evaluating f from every node's
    # coordinates (GMQ_EVAL_NODEWISE): the integrand as a whole at every
    # node, for comparison with the separable node sums of the timed steps
    nodewise = None
    if not args.no_nodewise_step:
        ctx.set_eval_mode(gmq.EVAL_NODEWISE)
        flush.fill_(1)
        torch.cuda.synchronize()
        e0.record(stream)
        nw_regions, _ = step()
        e1.record(stream)
        torch.cuda.synchronize()
        ctx.set_eval_mode(gmq.EVAL_SEPARABLE)
        nw_ms = e0.elapsed_time(e1)
        nodewise = {"value": nw_regions / (nw_ms / 1000.0), "unit": UNIT, "ms_per_step": nw_ms,
                    "regions_per_step": nw_regions,
                    "note": "one step of the same workload with GMQ_EVAL_NODEWISE (f from every "
                            "node's coordinates), timed like the e2e step"}
    tt = time_to_tol(ctx, stream, 1e-6) if not args.no_time_to_tol else None

    ms_step = total_ms / args.steps
    my_time, my_regions = aggregate_over_ranks(total_ms / 1000.0, regions, ws,
                                               f"cuda:{dev}" if ws > 1 else "cpu")
    value = my_regions / my_time
    if rank != 0:
        return
    rule = prof["rule"]
    # FP64 roofline of the rule kernel: FP64 instructions (and flops) per
    # region of each family at d = 8 (a fixed count: the integrand at 401
    # nodes plus one accumulation each and the per-region epilogue) times the
    # regions of that family in the timed steps, over the rule kernel's
    # event-timed launches.  Peak: the measured FP64 FMA issue rate (probe
    # kernel, same process); beside it the nominal 2 FP64 lanes per clock per
    # SM (1.25 TFLOP/s / 2 / 152 SMs / 2.07 GHz) at the median SM clock.
    roof = None
    clocks = clk.summary()
    counts_current = rule_source_fingerprint() == RULE_COUNTS_SHA16
    if rule["launches"] and all(f in RULE_FP64_INST_D8 for f in timed_fam_regions):
        n_launch = rule["launches"]
        avg_s = rule["ms"] / 1000.0 / n_launch
        inst = sum(RULE_FP64_INST_D8[f] * n for f, n in timed_fam_regions.items()) / n_launch
        flops = sum(RULE_FP64_FLOPS_D8[f] * n for f, n in timed_fam_regions.items()) / n_launch
        mhz = clocks.get("sm_mhz") or 2070.0
        peak_nominal = 2 * 152 * mhz * 1e6 / 1e9  # G FP64 lane-inst/s
        peak = probe64 / 1e9
        ach = inst / avg_s / 1e9
        roof = {"bound": "alu", "achieved": ach, "peak": peak,
                "unit": "G FP64 lane-inst/s", "frac": ach / peak if counts_current else None,
                "traffic": (RULE_DRAM_BYTES_PER_REGION_D8 * rule["regions"] / n_launch
                            if counts_current else None),
                "kernel": "k_rule64 (FP64 rule evaluation)",
                "peak_basis": ("measured: fastest FP64 chain of the issue-rate probe "
                               "(gmq_probe_fp_rate, 64 warps/SM, 16 independent chains per "
                               f"thread) in this run, median {probe_clocks.get('sm_mhz')} MHz"),
                "probe_G_lane_ops_per_s": {k: v / 1e9 for k, v in probe_ops.items()},
                "nominal": {"peak": peak_nominal, "frac": ach / peak_nominal,
                            "basis": (f"2 FP64 lanes/clk/SM (1.25 TFLOP/s nominal) x 152 SMs "
                                      f"x median {mhz:.0f} MHz")},
                "counts_match_source": counts_current,
                "flops_view": {"achieved_gflops": flops / avg_s / 1e9,
                               "peak_gflops_measured_fma": 2 * probe_ops["fma"] / 1e9},
                "inst_per_region": {G.FAMILY_NAMES[f]: RULE_FP64_INST_D8[f]
                                    for f in sorted(timed_fam_regions)},
                "regions_by_family": {G.FAMILY_NAMES[f]: n // args.steps
                                      for f, n in sorted(timed_fam_regions.items())}}
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
        "nodewise_step": nodewise,
        "unprofiled_step": {"ms": unprofiled_ms, "timed_ms_per_step": total_ms / args.steps,
                            "note": "the e2e step, per-launch timing events off"},
        "roofline": roof,
        "roofline_mixed": roof_mixed,
        "rule_eval_modes": modes,
        "e2e": {"value": e2e_regions / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": len(probs) * 4 * 8 * 8,
                "d2h_bytes_per_step": e2e_sweeps * 80},
        "clocks": clocks,
        "time_to_1e-6": tt,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
