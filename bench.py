"""Benchmark: OPF solves/s of the 123-bus synthetic feeder (single instance).

One step = one complete solve through the library, inputs resident on the
device: the Algorithm 1 precomputation (Sec. III-B) followed by ADMM
iterations to the stopping test (Sec. III-C with eps_rel = 1e-8 and
pres <= 1e-4, which puts the objective within 1e-6 of the LP optimum) and the
read-back of the objective.  The default path iterates in FP32 with one warp
per subsystem inside one thread-block cluster, re-centred in FP64, followed
by an FP64 polish;
``--precision fp64`` times plain FP64 iterations.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the library's stream, with a write of a 512 MiB buffer (larger than the
129 MB L2) between steps; barrier + synchronize on both sides; the maximum
over ranks.  Under torchrun every rank solves its own replica (no collective
on the data path: scaling "weak").

Extra fields: ``e2e`` (the same metric through the C ABI from host arrays,
host->device upload and device->host read of x inside the timed region),
``roofline`` of the dominant kernel, ``clocks`` sampled by nvidia-smi during
the timed region, ``cpu_baseline`` (the FP64 CPU oracle on this host), and
``gpu_launches``.

``--impl reference`` times the CPU oracle (plain FP64 C loop of Algorithm 1,
one core) on the same workload and prints the same line with
``"impl": "reference"``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "123"
SEED = 2001
RHO, EPS_REL, EPS_ABS = 100.0, 1e-8, 1e-4
METRIC = "OPF solves/s to 1e-4 residual (batched/served vs plain FP64); p50/p99 latency"
UNIT = "solves/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def workload_config(precision):
    return {
        "workload": "123-bus synthetic radial 3-phase feeder (seed 2001), single instance, "
                    "85 loads, 10 DERs, rho=100, stop at eps_rel=1e-8 and pres<=1e-4",
        "buses": 123,
        "precision": precision,
        "step": "precompute + ADMM iterations to the stopping test + objective read-back",
        "l2": "512 MiB buffer written between timed steps (working set ~1 MB < L2)",
        "parallelism": "replicas",
    }


def feeder():
    from paper_2310_09410_gb300 import synth
    return synth.preset_feeder(WORKLOAD, SEED)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except ValueError:
                continue
            for name, v in zip(names[1:], r[4:8]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes_per_iter(sizes, w):
    """Minimum bytes one iteration must move: each factor entry once, per slot
    lambda and x_s read+write, bbar read, u written and read (7 words), three
    index words (global, u position, segment start+count: 16 bytes), per global
    cost and both bounds (3 words)."""
    return w * (sizes["sum_nf"] + 7 * sizes["n_slots"] + 3 * sizes["n_global"]) + 16 * sizes["n_slots"]


def measured_peak():
    try:
        with open(PEAKS) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(f, budget_s=15.0):
    """FP64 CPU oracle, one thread, on a bounded sample of the same workload."""
    from oracle import admm as oracle_admm, lindist
    t0 = time.perf_counter()
    n = 0
    iters = 0
    while True:
        M = lindist.build(f)
        P = oracle_admm.Prepared(M)
        r = oracle_admm.admm(P, rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, max_iter=2_000_000,
                             check_every=50)
        n += 1
        iters += r.iters
        el = time.perf_counter() - t0
        if el >= budget_s or n >= 50:
            break
    return {"value": n / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} full solves of the same 123-bus instance (LP build, precompute, "
                      f"{iters // n} iterations each) in {el:.1f} s, plain FP64 C loop, one thread"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    f = feeder()
    from oracle import admm as oracle_admm, lindist

    def one():
        M = lindist.build(f)
        P = oracle_admm.Prepared(M)
        return oracle_admm.admm(P, rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS,
                                max_iter=2_000_000, check_every=50)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = one()
    el = time.perf_counter() - t0
    value = args.steps / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config("fp64 (CPU oracle)"), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full solves ({r.iters} iterations each), one thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# DRAM bytes of one k_warp_engine launch (1000 iterations) from the ncu
# capture in profiles/k_warp_engine_123bus.md; null for other kernels.
WARP_ENGINE_TRAFFIC_PER_LAUNCH = 352256 + 1536
ITERS_PER_LAUNCH = 1000


def max_over_ranks(value: float, world: int, device) -> float:
    """Largest value over the ranks (the timing reduction of the replicas)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def count_launches(stats, precision, k=50, R=1000):
    """Kernels of ours per step: precompute (3) + solve + objective read (1)."""
    n = 3 + 1
    if precision == "fp64":
        return n + 1 + (stats["main_iters"] // k) * (k + 1)
    main, pol = stats["main_iters"], stats["polish_iters"]
    bodies = -(-main // R)
    return n + 8 + bodies * 7 + 1 + 1 + (pol // k) * (k + 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="launch the iteration kernels directly instead of one graph with a device WHILE "
                         "node (same kernels and arithmetic; profilers cannot see kernels in such graphs)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_09410_gb300 import opf

    f = feeder()
    prec = opf.PREC_MIXED if args.precision == "mixed" else opf.PREC_FP64
    stream = torch.cuda.Stream(device=local)
    solver = opf.Solver.from_feeder(f, device=local, stream=stream.cuda_stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    flags = opf.SOLVE_HOST_LOOP if args.host_loop else 0

    def step():
        solver.precompute()
        ok = solver.solve(rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, precision=prec, flags=flags)
        _, obj = solver.solution()
        return ok, obj

    for _ in range(args.warmup):
        step()
    solver.precompute()
    sizes = solver.sizes()            # factor sizes are known after the precomputation
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times, objs, iters, iter_ms, launches = [], [], [], [], 0
    it_main, it_pol = 0, 0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ok, obj = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        objs.append(obj)
        st = solver.timing()
        iters.append(solver.residuals()["iters"])
        iter_ms.append(st["iterate_ms"])
        it_main += st["main_iters"]
        it_pol += st["polish_iters"]
        launches += count_launches(st, args.precision)
        if not ok:
            raise SystemExit("a timed solve did not converge")
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(float(sum(times)), world, f"cuda:{local}")
    value = world * args.steps / (total_ms / 1e3)

    # end to end through the C ABI from host arrays (create, precompute, solve, read x)
    e2e_times = []
    h2d = d2h = 0
    for _ in range(max(3, args.steps // 4)):
        t0 = time.perf_counter()
        s2 = opf.Solver.from_feeder(f, device=local, stream=stream.cuda_stream)
        s2.precompute()
        s2.solve(rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, precision=prec, flags=flags)
        x, obj = s2.solution()
        e2e_times.append(time.perf_counter() - t0)
        h2d = s2.sizes()["h2d_bytes"]
        d2h = x.nbytes + 8
        s2.close()
    e2e_total = max_over_ranks(sum(e2e_times), world, f"cuda:{local}")
    e2e_value = world * len(e2e_times) / e2e_total

    # roofline of the dominant kernel: the iteration phase (one-CTA engine or grid iterations)
    w = 4 if args.precision == "mixed" else 8
    bpi = algorithmic_bytes_per_iter(sizes, w)
    n_it = it_main if args.precision == "mixed" else sum(iters)
    achieved = bpi * n_it / (sum(iter_ms) / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    mixed = args.precision == "mixed"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": WARP_ENGINE_TRAFFIC_PER_LAUNCH if mixed else None,
            "traffic_unit": "bytes per launch of %d iterations" % ITERS_PER_LAUNCH if mixed else None,
            "algorithmic_bytes_per_launch": bpi * ITERS_PER_LAUNCH if mixed else None,
            "kernel": "k_warp_engine (FP32 iterations; one warp per subsystem, factors in registers, "
                      "instance resident in one thread-block cluster)"
            if args.precision == "mixed" else "k_tile_iter<double> (FP64 iterations, one CTA per tile)",
            "bytes_per_iter": bpi, "iters_timed": n_it, "peak_source": peak_kind + " hbm_gbs"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if args.precision == "mixed" else "f64",
                "data": "synthetic", "config": workload_config(args.precision),
                "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
                "iterations": {"mean": float(np.mean(iters)), "main": it_main // args.steps,
                               "polish": it_pol // args.steps},
                "objective": float(np.mean(objs)),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "roofline": roof, "clocks": clocks, "gpu_launches": int(launches)}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(f)
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
