"""Benchmark: OPF solves/s on one GB300.

Default workload (``--workload batch``): 1024 load scenarios of the 123-bus
synthetic feeder (seed 2001; scenario j scales every load by U[0.6, 1.2] x
N(1, 0.05) from seed 4000 + j), all solved together by the batched engine.
One step = one pass of the whole path over the batch, inputs resident on the
device: the feeder's FP64 factorization (Sec. III-B), the per-scenario
bbar = A_s^+ b, ADMM iterations of every instance to its own stopping test
(Sec. III-C with eps_rel = 1e-8 and pres <= 1e-4; FP32 iterations re-centred
in FP64, then an FP64 polish) and the read-back of the 1024 objectives.  The
same line reports the plain single-instance FP64 GPU path on the feeder
(``plain_fp64``) that the metric compares against.

``--workload single`` times one instance of the 123-bus feeder per step
(``--precision fp64`` for plain FP64 iterations).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the library's stream, with a write of a 512 MiB buffer (larger than the
129 MB L2) between steps; barrier + synchronize on both sides; the maximum
over ranks.  Under torchrun every rank solves its own replica (no collective
on the data path: scaling "weak").

Extra fields: ``e2e`` (the same metric through the C ABI from host arrays,
host->device upload of the loads and device->host read of x and the
objectives inside the timed region), ``roofline`` of the dominant kernel,
``clocks`` sampled by nvidia-smi during the timed region, ``cpu_baseline``
(the FP64 CPU oracle on this host, one thread, on a bounded sample) and
``gpu_launches``.

``--impl reference`` times the CPU oracle (plain FP64 C loop of Algorithm 1,
one thread) on the same workload, one scenario per step, and prints the same
line with ``"impl": "reference"``.
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

FEEDER, SEED = "123", 2001
# single-instance workloads: the 13-, 123- and 8500-bus configurations (and the
# 34-bus feeder of the serving mix)
SINGLE_SEEDS = {"13": 1001, "34": 5034, "123": 2001, "8500": 3001}
# Sec. III-C relative tolerance per feeder: the large feeder's norms run over
# ~1.1e5 slots, and eps_rel = 1e-8 there leaves the objective 2.9e-6 away
# from the LP optimum; 2e-9 gives 2.5e-7
SINGLE_EPS_REL = {"13": 1e-8, "34": 1e-8, "123": 1e-8, "8500": 2e-9}
N_SCEN, SCEN_SEED0 = 1024, 4000
RHO, EPS_REL, EPS_ABS = 100.0, 1e-8, 1e-4
# Iterations between stopping tests of the batched workload.  A test
# iteration of the batched engine costs about two ordinary ones; on the 1024 x
# 123-bus batch 50 and 100 gave the same stopping iterations for every
# instance (the FP32 phase met the test only at multiples of 100), with the
# FP32 phase 207.5 and 202.2 ms; 20 / 200 gave 220.6 / 199.6 ms with 22 fewer
# / 24 more iterations on average.
BATCH_CHECK_EVERY = 100
METRIC = "OPF solves/s to 1e-4 residual (batched/served vs plain FP64); p50/p99 latency"
UNIT = "solves/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")

# FP32 lanes per SM (Blackwell: 4 sub-partitions x 32), for the nominal FP32
# SIMT peak printed beside the measured one; the SM count and the clock are
# read from the device and from the clock samples of the run.
FP32_LANES = 128

# DRAM bytes per launch of the dominant kernels, copied from the ncu captures
# summarised in profiles/ (a copied constant, labelled so in the line; None
# once the kernel has changed since the capture).
BATCH_ENGINE_TRAFFIC_PER_LAUNCH = 63054592 + 893184
BATCH_ENGINE_TRAFFIC_SOURCE = "profiles/k_batch_engine_123bus_x1024.md"
# Warp instructions per instance-iteration of the batched engine in the
# shape the autotune picks for the 1024 x 123-bus batch (8 instances per CTA,
# 16 warps, tensor memory): smsp__inst_executed.sum of the same capture over
# its 4000 iterations x 1024 instances (copied; None for other shapes).
BATCH_ENGINE_INST_PER_INSTANCE_ITER = 16.7984e9 / (4000 * 1024)
BATCH_ENGINE_INST_SHAPE = {"k_inst": 8, "warps": 16, "tmem": 1}
WARP_ENGINE_TRAFFIC_PER_LAUNCH = 516864 + 768
PERSIST_ENGINE_TRAFFIC_PER_LAUNCH = 8708352 + 313088
ITERS_PER_LAUNCH = 1000


def issue_roofline(shape, inst_iters, engine_ms, sm_mhz):
    """Instruction-issue figure of the batched engine (its bound): warp
    instructions issued per cycle on each SM of its grid against the 4 an SM
    issues at most, from the instructions per instance-iteration of the ncu
    capture and this run's instance-iterations, engine time and SM clock."""
    if any(shape.get(k) != v for k, v in BATCH_ENGINE_INST_SHAPE.items()) or not engine_ms:
        return None
    inst = BATCH_ENGINE_INST_PER_INSTANCE_ITER * inst_iters
    ipc = inst / (engine_ms / 1e3 * sm_mhz * 1e6 * shape["ctas"])
    return {"achieved_ipc_per_sm": ipc, "peak_ipc_per_sm": 4.0, "frac": ipc / 4.0, "sms": shape["ctas"],
            "sm_mhz": sm_mhz,
            "warp_instructions_per_instance_iteration": BATCH_ENGINE_INST_PER_INSTANCE_ITER,
            "source": "instructions per instance-iteration copied from the ncu capture in "
                      + BATCH_ENGINE_TRAFFIC_SOURCE + " (smsp__inst_executed.sum, not measured in this run); "
                      "instance-iterations, engine time and SM clock measured in this run"}


def batch_config(n):
    return {
        "workload": f"{n} load scenarios of the 123-bus synthetic radial 3-phase feeder (seed 2001; "
                    "85 loads scaled by U[0.6,1.2] x N(1,0.05) per scenario, seeds 4000+j), 10 DERs, "
                    f"rho=100, each instance stopped at eps_rel=1e-8 and pres<=1e-4 (Sec. III-C test every "
                    f"{BATCH_CHECK_EVERY} iterations)",
        "buses": 123, "instances": n, "precision": "FP32 iterations re-centred in FP64 + FP64 polish",
        "step": "factorization of the feeder (FP64) + per-scenario bbar = A_s^+ b + ADMM to the test "
                "for every instance + objectives read back",
        "l2": "512 MiB buffer written between timed steps",
        "parallelism": "replicas",
    }


SINGLE_SHAPE = {"13": "12 lines, 2 DERs", "34": "33 lines", "123": "85 loads, 10 DERs",
                "8500": "1200 loads, 100 DERs, tree depth <= 60"}


def single_config(precision, name="123", fixed_iters=0):
    stop = (f"exactly {fixed_iters} iterations (profiling run, no stopping test)" if fixed_iters else
            f"stop at eps_rel={SINGLE_EPS_REL[name]:g} and pres<=1e-4")
    return {
        "workload": f"{name}-bus synthetic radial 3-phase feeder (seed {SINGLE_SEEDS[name]}), single instance, "
                    f"{SINGLE_SHAPE[name]}, rho=100, {stop}",
        "buses": int(name), "precision": precision,
        "step": "precompute + ADMM iterations to the stopping test + objective read-back",
        "l2": "512 MiB buffer written between timed steps",
        "parallelism": "replicas",
    }


def feeder():
    from paper_2310_09410_gb300 import synth
    return synth.preset_feeder(FEEDER, SEED)


def scenario_loads(f, n):
    from paper_2310_09410_gb300 import synth
    fs = [synth.load_scenario(f, SCEN_SEED0 + j) for j in range(n)]
    return fs, np.stack([g["load_a"] for g in fs]), np.stack([g["load_b"] for g in fs])


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
    """Minimum bytes one single-instance iteration must move: each factor entry
    once, per slot lambda and x_s read+write, bbar read, u written and read (7
    words), three index words (16 bytes), per global cost and both bounds."""
    return w * (sizes["sum_nf"] + 7 * sizes["n_slots"] + 3 * sizes["n_global"]) + 16 * sizes["n_slots"]


def algorithmic_flops_per_iter(sizes):
    """Flops of one iteration of one instance: the two products with the
    factor (2 flops per entry each), 8 per slot (v, x_s, lambda, u and the
    copy's share of the segment sum) and 2 per global (shift and scale)."""
    return 4 * sizes["sum_nf"] + 8 * sizes["n_slots"] + 2 * sizes["n_global"]


def measured_peak():
    try:
        with open(PEAKS) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def fp32_fma_peak(opf, torch, device, stream, reps=10):
    """FP32 FMA throughput of the device measured now: the library's FMA probe
    (8 independent chains per thread, two 1024-thread CTAs per SM) timed with
    CUDA events on `stream`; median and best of `reps` launches."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, threads, iters = 2 * sms, 1024, 2048
    out = torch.empty(blocks * threads, dtype=torch.float32, device=torch.device("cuda", device))
    torch.cuda.synchronize()
    for _ in range(3):
        opf.probe_fma(blocks, threads, iters, out.data_ptr(), stream.cuda_stream)
    times, fl = [], 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = opf.probe_fma(blocks, threads, iters, out.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    med, best = statistics.median(times), min(times)
    return {"tflops": fl / (med / 1e3) / 1e12, "tflops_best": fl / (best / 1e3) / 1e12, "sms": sms,
            "flops_per_launch": fl, "ms_median": med, "launches": reps}


def fp64_fma_peak(opf, torch, device, stream, reps=5):
    """FP64 FMA throughput of the device measured now (`opf_probe_dfma`), for
    the FP64 iterations' ALU fraction; median of `reps` launches."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks, threads, iters = 2 * sms, 1024, 32
    out = torch.empty(blocks * threads, dtype=torch.float64, device=torch.device("cuda", device))
    torch.cuda.synchronize()
    opf.probe_dfma(blocks, threads, iters, out.data_ptr(), stream.cuda_stream)
    times, fl = [], 0.0
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = opf.probe_dfma(blocks, threads, iters, out.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return fl / (statistics.median(times) / 1e3) / 1e12


def _lp_optimum(g):
    """The oracle's LP optimum of one instance (pool worker)."""
    from oracle import admm as oracle_admm, lindist
    return oracle_admm.lp_optimum(lindist.build(g))[0]


def oracle_error(instances, objs, pres_gpu, x=None, locals_of=None, sample=64):
    """Error of every result against the FP64 oracle (part of the CPU-baseline
    leg): relative objective error of each instance against the oracle's LP
    optimum of that instance (computed on spawned host processes), and pres
    recomputed on the host from the library's x and local copies x_s for a
    sample of instances, |x[g(k)] - x_s,k| stacked over the slots."""
    import multiprocessing as mp
    from oracle import lindist
    t0 = time.perf_counter()
    cores = min(_host_cores(), 16, len(instances))
    if cores > 1:
        with mp.get_context("spawn").Pool(cores) as pool:
            star = np.array(pool.map(_lp_optimum, instances, chunksize=max(1, len(instances) // (4 * cores))))
    else:
        star = np.array([_lp_optimum(g) for g in instances])
    rel = np.abs(np.asarray(objs) - star) / np.abs(star)
    out = {"max_obj_rel": float(rel.max()), "mean_obj_rel": float(rel.mean()), "instances": len(instances),
           "max_pres": float(np.max(pres_gpu)),
           "reference": "LP optimum of each instance (oracle: HiGHS on the centralized LP of Eq. LP_model)"}
    if x is not None and locals_of is not None:
        # canonical slot -> global index (the instances share one topology)
        gidx = np.concatenate([sb["idx"] for sb in lindist.build(instances[0]).subs])
        picks = np.unique(np.linspace(0, len(instances) - 1, min(sample, len(instances))).astype(int))
        ph, dif = [], []
        for j in picks:
            xs, _ = locals_of(int(j))
            p = float(np.linalg.norm(x[j][gidx] - xs))
            ph.append(p)
            dif.append(abs(p - float(pres_gpu[j])) / max(float(pres_gpu[j]), 1e-300))
        out.update({"max_pres_host": max(ph), "pres_host_vs_gpu_max_rel_diff": max(dif),
                    "pres_host_sample": int(len(picks))})
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def oracle_solve(g):
    from oracle import admm as oracle_admm, lindist
    M = lindist.build(g)
    P = oracle_admm.Prepared(M)
    return oracle_admm.admm(P, rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, max_iter=2_000_000, check_every=50)


def _oracle_iters(g):
    """One oracle solve in a pool worker (module level, so a spawned worker can import it)."""
    return int(oracle_solve(g).iters)


def _host_cores():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return max(1, os.cpu_count() or 1)


def oracle_pool_solves(instances, n_proc, budget_s, start=0):
    """Independent oracle solves of the instances on n_proc spawned processes
    (one thread each), in waves of n_proc, until budget_s has passed.
    Returns (solves, iterations, seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")      # never fork a process that holds a CUDA context
    with ctx.Pool(n_proc) as pool:
        pool.map(_oracle_iters, [instances[(start + j) % len(instances)] for j in range(n_proc)])   # warm
        t0 = time.perf_counter()
        n = iters = 0
        k = start + n_proc
        while True:
            res = pool.map(_oracle_iters, [instances[(k + j) % len(instances)] for j in range(n_proc)])
            k += n_proc
            n += len(res)
            iters += sum(res)
            el = time.perf_counter() - t0
            if el >= budget_s:
                return n, iters, el


def cpu_baseline(instances, budget_s=15.0, what="scenarios of the batch"):
    """The FP64 CPU oracle on a bounded sample of the same workload: one
    thread for about a third of the budget, then (independent instances
    only) one process per host core for the rest."""
    t0 = time.perf_counter()
    n = iters = 0
    while True:
        r = oracle_solve(instances[n % len(instances)])
        n += 1
        iters += r.iters
        el = time.perf_counter() - t0
        if el >= budget_s / 3 or n >= 50:
            break
    one = n / el
    cores = _host_cores()
    if len(instances) < 2 or cores < 2:
        return {"value": one, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{n} full solves ({what}: LP build, precompute, {iters // n} iterations each on "
                          f"average) in {el:.1f} s, plain FP64 C loop, one thread"}
    m, it2, el2 = oracle_pool_solves(instances, cores, 2 * budget_s / 3, start=n)
    return {"value": m / el2, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} full solves ({what}: LP build, precompute, {it2 // m} iterations each on average) "
                      f"in {el2:.1f} s on {cores} processes, one per host core, one thread each (plain FP64 C "
                      f"loop); one core alone: {one:.3f} solves/s ({n} solves in {el:.1f} s)"}


def cpu_baseline_extrapolated(f, gpu_iters, budget_s=15.0, copied=False):
    """The oracle's per-iteration time on the instance, measured over a bounded
    number of iterations, times the iterations the GPU solve needed, plus its
    precompute: a full solve of the large feeder takes the CPU loop hours."""
    from oracle import admm as oracle_admm, lindist
    t0 = time.perf_counter()
    P = oracle_admm.Prepared(lindist.build(f))
    t_pre = time.perf_counter() - t0
    n = 200
    while True:
        t1 = time.perf_counter()
        oracle_admm.admm(P, rho=RHO, max_iter=n, check_every=50)
        el = time.perf_counter() - t1
        if el >= 0.25 * budget_s or n >= 1_000_000:
            break
        n *= 2
    per_it = el / n
    t_solve = t_pre + per_it * gpu_iters
    return {"value": 1.0 / t_solve, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"LP build + precompute ({t_pre:.1f} s) and {n} iterations ({per_it * 1e3:.3f} ms each) "
                      f"of the plain FP64 C loop, one thread, extrapolated to the {gpu_iters} iterations of the "
                      f"GPU solve" + (" (a copied constant: the count of an earlier GPU solve)" if copied else "")}


# Iterations of the 8500-bus solve at its stopping rule, copied from a GPU
# solve (FP32 iterations + FP64 polish; tests/test_large_gpu.py runs the same
# solve): the CPU reference arm extrapolates its per-iteration time to this
# count instead of running the hours-long loop, and says so in its line.
ITERS_8500 = 2_196_200


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    f = feeder()
    if args.workload == "single" and args.feeder == "8500":
        from paper_2310_09410_gb300 import synth
        cb = cpu_baseline_extrapolated(synth.preset_feeder("8500", SINGLE_SEEDS["8500"]), ITERS_8500, copied=True)
        value = cb["value"]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": 1,
                "warmup": 0, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": single_config("fp64 (CPU oracle)", "8500"), "impl": "reference",
                "cpu_baseline": cb,
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "single":
        from paper_2310_09410_gb300 import synth
        f = synth.preset_feeder(args.feeder, SINGLE_SEEDS[args.feeder])
    if args.workload == "batch":
        fs, _, _ = scenario_loads(f, max(args.steps + args.warmup, 1))
        config = batch_config(N_SCEN)
        what = "one scenario of the batch per step"
    else:
        fs = [f]
        config = single_config("fp64 (CPU oracle)", args.feeder)
        what = "the instance"
    cores = _host_cores() if args.workload == "batch" else 1
    if cores > 1:
        # one step: one scenario per host core, solved side by side by
        # spawned processes (the scenarios are independent)
        import multiprocessing as mp
        fs, _, _ = scenario_loads(f, max((args.steps + args.warmup) * cores, 1))
        what = f"{cores} scenarios of the batch per step, one per host core"
        with mp.get_context("spawn").Pool(cores) as pool:
            for j in range(args.warmup):
                pool.map(_oracle_iters, fs[j * cores:(j + 1) * cores])
            t0 = time.perf_counter()
            iters = 0
            for j in range(args.warmup, args.warmup + args.steps):
                iters += sum(pool.map(_oracle_iters, fs[j * cores:(j + 1) * cores]))
            el = time.perf_counter() - t0
        value = args.steps * cores / el
        iters //= cores
    else:
        for j in range(args.warmup):
            oracle_solve(fs[j % len(fs)])
        t0 = time.perf_counter()
        iters = 0
        for j in range(args.steps):
            iters += oracle_solve(fs[(args.warmup + j) % len(fs)]).iters
        el = time.perf_counter() - t0
        value = args.steps / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps ({what}, {iters // max(args.steps, 1)} "
                                       f"iterations per solve on average), one thread per process"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(value: float, world: int, device) -> float:
    """Largest value over the ranks (the timing reduction of the replicas)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def warp_engine_fp64(sizes):
    """The library's automatic choice runs FP64 iterations on the warp engine
    for instances of at most 64 subsystems of at most 64 slots."""
    return sizes["n_sub"] <= 64 and sizes["max_ns"] <= 64


def count_launches_single(stats, precision, k=50, R=1000, persistent=False, warp64=False, per_launch=20000):
    """Kernels of ours per single-instance step: precompute (3) + solve + objective read (1).
    FP64 iterations: the warp engine (one launch) for small instances, else the
    persistent engine (one launch per 20000 iterations); whole-grid kernels
    (k + 1 per chunk of k) only where neither holds the instance."""
    n = 3 + 1

    def fp64(iters):
        if warp64:
            return 1 + 1
        return 1 + (-(-iters // per_launch) if persistent else (iters // k) * (k + 1))
    if precision == "fp64":
        return n + fp64(stats["main_iters"])
    main, pol = stats["main_iters"], stats["polish_iters"]
    bodies = -(-main // R)
    return n + 8 + bodies * 7 + 1 + fp64(pol)


def count_launches_batch(t):
    """Kernels of ours per batched step: factorization (3) and A_s^+ (1), rhs
    and bbar (4), six per loop pass (re-centring 2, engine, unshift 2, loop
    test), the polish restart and objective (2), objective read (1)."""
    return 3 + 1 + 4 + 6 * (t["fp32_passes"] + t["fp64_passes"]) + 2 + 1


# Single-instance configurations reported beside the batch: (feeder, precision,
# timed solves); one untimed solve first (graph and engine plans).
SINGLE_RECORDS = (("13", "fp64", 20), ("13", "mixed", 20), ("123", "fp64", 3), ("123", "mixed", 5),
                  ("8500", "mixed", 1))


def single_records(opf, synth, device, stream):
    """Plain FP64 and FP32 + FP64-polish solves of single instances (the
    13-, 123- and 8500-bus configurations), each timed with CUDA events on the
    library's stream around precompute + solve + read-back."""
    import torch
    out = {}
    for name, prec, n in SINGLE_RECORDS:
        f = synth.preset_feeder(name, SINGLE_SEEDS[name])
        s = opf.Solver.from_feeder(f, device=device, stream=stream.cuda_stream)
        p = opf.PREC_FP64 if prec == "fp64" else opf.PREC_MIXED
        kw = dict(rho=RHO, eps_rel=SINGLE_EPS_REL[name], eps_abs_pres=EPS_ABS, max_iter=6_000_000, precision=p)
        s.precompute()
        s.solve(**dict(kw, max_iter=2000) if name == "8500" else kw)       # plans, graphs
        times, ok = [], True
        for _ in range(n):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.precompute()
            ok &= s.solve(**kw)
            x, obj = s.solution()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        r = s.residuals()
        out[f"{name}_{prec}"] = {"solves_per_s": 1e3 * n / sum(times), "ms_per_solve": sum(times) / n,
                                 "iterations": int(r["iters"]), "objective": obj, "pres": r["pres"],
                                 "converged": bool(ok), "solves_timed": n}
        s.close()
    return out


def plain_fp64_reference(opf, f, device, stream, n=2):
    """Solves/s of the plain single-instance FP64 GPU path on the feeder."""
    import torch
    s = opf.Solver.from_feeder(f, device=device, stream=stream.cuda_stream)
    times = []
    for j in range(n + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.precompute()
        ok = s.solve(rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, precision=opf.PREC_FP64)
        s.solution()
        e1.record(stream)
        e1.synchronize()
        if j:                        # the first solve builds the graph
            times.append(e0.elapsed_time(e1))
        if not ok:
            raise SystemExit("the plain FP64 solve did not converge")
    iters = s.residuals()["iters"]
    t = s.timing()
    fpi = algorithmic_flops_per_iter(s.sizes())
    s.close()
    peak64 = fp64_fma_peak(opf, torch, device, stream)
    ach = fpi * iters / (t["iterate_ms"] / 1e3) / 1e12 if t["iterate_ms"] > 0 else None
    return {"value": 1e3 * len(times) / sum(times), "unit": UNIT, "iterations": int(iters),
            "fp64_alu": {"achieved_tflops": ach, "peak_tflops": peak64, "frac": ach / peak64 if ach else None,
                         "peak_source": "measured in this run: FP64 FMA probe (opf_probe_dfma)",
                         "note": "latency-bound: one instance's iteration is a chain of small dependent "
                                 "products and a grid barrier"},
            "path": "single instance, FP64 iterations on the engine opf_solve_ex picks (warp engine up to 64 "
                    "subsystems, else the persistent grid engine)"}


def run_batch(args, rank, world, local):
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_09410_gb300 import opf, synth

    n = args.instances
    f = feeder()
    fs, lp, lq = scenario_loads(f, n)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=local)
    dlp = torch.from_numpy(lp).to(dev)
    dlq = torch.from_numpy(lq).to(dev)
    torch.cuda.synchronize()
    solver = opf.Solver.from_feeder(f, device=local, stream=stream.cuda_stream)
    solver.precompute()
    batch = opf.Batch(solver, n)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flags = opf.SOLVE_HOST_LOOP if args.host_loop else 0

    def step():
        solver.precompute()
        batch.set_loads_device(0, n, dlp.data_ptr(), dlq.data_ptr())
        ok = batch.solve(rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, check_every=BATCH_CHECK_EVERY,
                         precision=opf.PREC_MIXED, flags=flags)
        _, obj = batch.solution()
        return ok, obj

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times, launches, iters, objs = [], 0, [], None
    fp32_ms = fp64_ms = 0.0
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ok, objs = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        t = batch.timing()
        fp32_ms += t["fp32_ms"]
        fp64_ms += t["fp64_ms"]
        launches += count_launches_batch(t)
        iters.append(t["mean_iters"])
        if not ok:
            raise SystemExit("an instance of a timed batch did not converge")
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(float(sum(times)), world, f"cuda:{local}")
    value = world * n * args.steps / (total_ms / 1e3)
    st = batch.status()

    # end to end from pinned host arrays: loads uploaded, x and objectives read back
    lp_pin = torch.from_numpy(np.ascontiguousarray(lp)).pin_memory()
    lq_pin = torch.from_numpy(np.ascontiguousarray(lq)).pin_memory()
    x_pin = torch.empty((n, batch.n_global), dtype=torch.float64).pin_memory()
    obj_pin = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_times = []
    for _ in range(max(2, args.steps // 2)):
        t0 = time.perf_counter()
        solver.precompute()
        batch.set_loads(0, lp_pin.numpy(), lq_pin.numpy())
        batch.solve(rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, check_every=BATCH_CHECK_EVERY,
                    precision=opf.PREC_MIXED, flags=flags)
        x, _ = batch.solution(out=(x_pin.numpy(), obj_pin.numpy()))
        e2e_times.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(sum(e2e_times), world, f"cuda:{local}")
    e2e_value = world * n * len(e2e_times) / e2e_total
    h2d = lp.nbytes + lq.nbytes
    d2h = x.nbytes + 8 * n

    # dominant kernel: the FP32 engine, timed alone on direct launches
    solver.precompute()
    batch.set_loads_device(0, n, dlp.data_ptr(), dlq.data_ptr())
    batch.solve(rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, check_every=BATCH_CHECK_EVERY,
                precision=opf.PREC_MIXED, flags=opf.SOLVE_HOST_LOOP)
    th = batch.timing()
    sizes = solver.sizes()
    fpi = algorithmic_flops_per_iter(sizes)
    st_h = batch.status()
    x_h, obj_h = batch.solution()        # same inputs as the timed steps: the results checked against the oracle
    inst_iters = float(np.sum(st_h["iters"]))
    passes = max(th["fp32_passes"], 1)
    achieved = fpi * inst_iters / (th["engine_ms"] / 1e3) / 1e12 if th["engine_ms"] > 0 else None
    probe = fp32_fma_peak(opf, torch, local, stream)
    peak = probe["tflops"]
    max_mhz = clocks.get("sm_max_mhz") or 2070.0
    nominal = probe["sms"] * FP32_LANES * 2 * max_mhz * 1e6 / 1e12
    shape = batch.shape(opf.PREC_FP32)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None,
            "peak_source": "measured in this run: FP32 FMA probe (opf_probe_fma, %d CTAs x 1024 threads, 8 "
                           "independent chains each), median of %d launches timed with CUDA events; best %.1f "
                           "TFLOP/s; nominal %d SMs x %d lanes x 2 x %.0f MHz = %.1f TFLOP/s"
                           % (2 * probe["sms"], probe["launches"], probe["tflops_best"], probe["sms"],
                              FP32_LANES, max_mhz, nominal),
            "frac_of_nominal": achieved / nominal if achieved else None,
            "traffic": BATCH_ENGINE_TRAFFIC_PER_LAUNCH,
            "traffic_unit": "DRAM bytes per engine launch of 4000 iterations, copied from the ncu capture in "
                            + BATCH_ENGINE_TRAFFIC_SOURCE + " (not measured in this run)",
            "kernel": "k_batch_engine<float> (FP32; %d instances per CTA, %d warps, %d CTAs; factors, u and x "
                      "in shared memory, lambda and bbar~ %s)"
                      % (shape["k_inst"], shape["warps"], shape["ctas"],
                         "in tensor memory (%d TMEM columns per CTA)" % shape["tmem_cols"] if shape["tmem"]
                         else "streamed from L2"),
            "issue": issue_roofline(shape, inst_iters, th["engine_ms"], clocks.get("sm_mhz") or max_mhz),
            "flops_per_instance_iteration": fpi,
            "instance_iterations_timed": inst_iters,
            "launches_timed": passes,
            "engine_ms": th["engine_ms"],
            "note": "instance iterations include those of the FP64 polish (%d pass(es), about 1%% of them), "
                    "so achieved is over-stated by about that much" % th["fp64_passes"]}

    plain = None if args.no_plain_fp64 else plain_fp64_reference(opf, f, local, stream)
    singles = single_records(opf, synth, local, stream) if args.single_records else None
    serve = None
    if args.serve_requests > 0:
        # the serving workload, short: the metric's p50/p99 latency per feeder class
        sr = serve_measure(args, local, args.serve_requests, 200, drain_s=args.max_service_s + 1.0)
        serve = {"value": sr["value"], "unit": UNIT, "p50_ms": sr["p50_ms"], "p99_ms": sr["p99_ms"],
                 "per_class": sr["per_class"], "window_s": sr["window_s"], "requests": sr["requests"],
                 "warm_requests": sr["warm_requests"], "clocks": sr["clocks"],
                 "config": dict(serve_config(args), workload=serve_config(args)["workload"].replace(
                     f"{args.requests} requests after", f"{args.serve_requests} requests after").replace(
                     f"at most {args.drain_s:.0f} s", f"at most {args.max_service_s + 1.0:.0f} s"))}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": batch_config(n),
                "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99)),
                               "note": "every instance of a batch returns with the batch"},
                "phases_ms": {"fp32": fp32_ms / args.steps, "fp64_polish": fp64_ms / args.steps},
                "iterations": {"mean": float(np.mean(iters)), "max": int(np.max(st["iters"])),
                               "min": int(np.min(st["iters"]))},
                "converged": int(np.sum(st["converged"])), "max_pres": float(np.max(st["pres"])),
                "objective_mean": float(np.mean(objs)),
                "plain_fp64": dict(plain, speedup=value / plain["value"]) if plain else None,
                "shape": shape, "tune_log": batch.tune_log(),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "roofline": roof, "clocks": clocks, "gpu_launches": int(launches)}
        if serve is not None:
            line["serve"] = serve
        if singles is not None:
            line["single"] = singles
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(fs)
            line["oracle_error"] = oracle_error(fs, obj_h, st_h["pres"], x=x_h, locals_of=batch.locals)
            if singles is not None:
                # the single-instance objectives against the oracle's LP optimum
                # (the 8500-bus LP takes the host about half a minute: not here)
                for key, rec in singles.items():
                    name = key.split("_")[0]
                    if name != "8500":
                        star = _lp_optimum(synth.preset_feeder(name, SINGLE_SEEDS[name]))
                        rec["obj_rel_err"] = abs(rec["objective"] - star) / abs(star)
        print(json.dumps(line), flush=True)
    batch.close()
    solver.close()
    return 0


def run_single(args, rank, world, local):
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_09410_gb300 import opf, synth

    name = args.feeder
    f = synth.preset_feeder(name, SINGLE_SEEDS[name])
    eps_rel = 0.0 if args.fixed_iters else SINGLE_EPS_REL[name]
    max_iter = args.fixed_iters if args.fixed_iters else 6_000_000
    prec = opf.PREC_MIXED if args.precision == "mixed" else opf.PREC_FP64
    stream = torch.cuda.Stream(device=local)
    solver = opf.Solver.from_feeder(f, device=local, stream=stream.cuda_stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    flags = opf.SOLVE_HOST_LOOP if args.host_loop else 0

    def step():
        solver.precompute()
        ok = solver.solve(rho=RHO, eps_rel=eps_rel, eps_abs_pres=EPS_ABS, max_iter=max_iter, precision=prec,
                          flags=flags)
        _, obj = solver.solution()
        return ok or bool(args.fixed_iters), obj

    for _ in range(args.warmup):
        step()
    solver.precompute()
    sizes = solver.sizes()
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
        launches += count_launches_single(st, args.precision, persistent=not warp_engine_fp64(sizes),
                                          warp64=warp_engine_fp64(sizes))
        if not ok:
            raise SystemExit("a timed solve did not converge")
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = max_over_ranks(float(sum(times)), world, f"cuda:{local}")
    value = world * args.steps / (total_ms / 1e3)

    e2e_times = []
    h2d = d2h = 0
    for _ in range(max(1 if name == "8500" else 3, args.steps // 4)):
        t0 = time.perf_counter()
        s2 = opf.Solver.from_feeder(f, device=local, stream=stream.cuda_stream)
        s2.precompute()
        s2.solve(rho=RHO, eps_rel=eps_rel, eps_abs_pres=EPS_ABS, max_iter=max_iter, precision=prec, flags=flags)
        x, obj = s2.solution()
        e2e_times.append(time.perf_counter() - t0)
        h2d = s2.sizes()["h2d_bytes"]
        d2h = x.nbytes + 8
        s2.close()
    e2e_total = max_over_ranks(sum(e2e_times), world, f"cuda:{local}")
    e2e_value = world * len(e2e_times) / e2e_total

    w = 4 if args.precision == "mixed" else 8
    bpi = algorithmic_bytes_per_iter(sizes, w)
    n_it = it_main if args.precision == "mixed" else sum(iters)
    achieved = bpi * n_it / (sum(iter_ms) / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    mixed = args.precision == "mixed"
    big = sizes["n_slots"] > 4096
    if mixed and not big:
        kern, traffic = ("k_warp_engine<float> (FP32 iterations; one warp per subsystem, factors in registers, "
                         "instance resident in one thread-block cluster)"), WARP_ENGINE_TRAFFIC_PER_LAUNCH
    elif big:
        kern = ("k_persist_engine<%s> (%s iterations; cooperative launch over two CTAs per SM, instance "
                "resident in their shared memory, one grid barrier per iteration)"
                % (("float", "FP32") if mixed else ("double", "FP64")))
        traffic = PERSIST_ENGINE_TRAFFIC_PER_LAUNCH if mixed else None
    elif warp_engine_fp64(sizes):
        kern, traffic = ("k_warp_engine<double> (FP64 iterations; one warp per subsystem, factors in shared "
                         "memory, instance resident in one thread-block cluster)"), None
    else:
        kern, traffic = ("k_persist_engine<double> (FP64 iterations; cooperative launch, instance resident in "
                         "the CTAs' shared memory, one grid barrier per iteration)"), None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": traffic,
            "traffic_unit": "bytes per launch of %d iterations" % ITERS_PER_LAUNCH if traffic else None,
            "algorithmic_bytes_per_launch": bpi * ITERS_PER_LAUNCH if mixed else None,
            "kernel": kern,
            "bytes_per_iter": bpi, "iters_timed": n_it, "peak_source": peak_kind + " hbm_gbs"}
    if not mixed:
        # FP64 iterations: the FP64 FMA rate measured now is the other ceiling
        peak64 = fp64_fma_peak(opf, torch, local, stream)
        ach64 = algorithmic_flops_per_iter(sizes) * n_it / (sum(iter_ms) / 1e3) / 1e12
        roof["fp64_alu"] = {"achieved_tflops": ach64, "peak_tflops": peak64, "frac": ach64 / peak64,
                            "peak_source": "measured in this run: FP64 FMA probe (opf_probe_dfma)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if mixed else "f64",
                "data": "synthetic", "config": single_config(args.precision, name, args.fixed_iters),
                "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
                "iterations": {"mean": float(np.mean(iters)), "main": it_main // args.steps,
                               "polish": it_pol // args.steps},
                "objective": float(np.mean(objs)),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "roofline": roof, "clocks": clocks, "gpu_launches": int(launches)}
        if world == 1 and not args.no_cpu_baseline:
            if name == "8500" or args.fixed_iters:
                line["cpu_baseline"] = cpu_baseline_extrapolated(f, int(np.mean(iters)))
            else:
                line["cpu_baseline"] = cpu_baseline([f], what="the same instance")
            if not args.fixed_iters:
                x1, _ = solver.solution()
                line["oracle_error"] = oracle_error([f], [objs[-1]], [solver.residuals()["pres"]],
                                                    x=x1[None, :], locals_of=lambda j: solver.locals())
        print(json.dumps(line), flush=True)
    solver.close()
    return 0


SERVE_SIZES = ("13", "34", "123", "8500")
SERVE_WEIGHTS = (0.4, 0.3, 0.2, 0.1)
SERVE_FEEDER_SEEDS = {"13": 5013, "34": 5034, "123": 5123, "8500": 5850}
SERVE_ARRIVAL_SEED, SERVE_REQ_SEED0, SERVE_RATE = 5000, 6000, 2000.0


def serve_config(args):
    return {
        "workload": f"serving: Poisson arrivals ({args.rate:.0f}/s, seed 5000) of solve requests, feeder mix "
                    f"13/34/123/8500 buses with weights {args.mix.replace(',', '/')} (topologies seeds "
                    f"5013/5034/5123/5850), request r with the load scenario of seed 6000+r; each request FP32 + "
                    f"FP64 polish to eps_rel=1e-8 (8500 buses: 2e-9) and pres<=1e-4; {args.requests} requests after "
                    f"{args.warm_requests} warm-up requests; arrivals stop after the last request, then the "
                    f"server drains for at most {args.drain_s:.0f} s",
        "admission": f"every model: a request whose predicted wait for a slot exceeds {args.max_wait_s:g} s is "
                     f"refused at submit, one that has waited longer is shed; 8500-bus requests stop after "
                     f"{args.max_service_s:g} s of service; each outcome is counted per class",
        "models": f"13/34/123-bus: continuous batching in the batched engine ("
                  + (f"FP32 shape {args.serve_k} instances per CTA, {args.serve_warps} warps: latency first"
                     if args.serve_k else "FP32 shape autotuned on a full batch") +
                  f"), passes of {args.chunk} FP32 iterations "
                  f"(slots in the FP64 polish: {args.polish_chunk or 100} FP64 iterations per pass); "
                  f"8500-bus: {args.big_handles} "
                  f"single-instance handles on worker threads, each on an SM partition of {args.big_sms} SMs "
                  f"(green context); the batched models on "
                  + ("the remaining SMs' partition" if args.batched_partition else "ordinary streams"),
        "parallelism": "replicas",
    }


def serve_measure(args, local, requests, warm_requests, drain_s):
    """The serving workload: Poisson arrivals of the feeder mix submitted to
    the request server, which admits, batches and retires them; each model
    has an admission policy (bounded wait for a slot, bounded service time),
    so every measured request ends served, refused at submit, shed from the
    queue or stopped at its service bound, each with its status counted.
    Returns the per-class and overall results."""
    import torch
    from paper_2310_09410_gb300 import opf, synth

    weights = np.array([float(w) for w in args.mix.split(",")])
    weights = weights / weights.sum()
    feeders = {k: synth.preset_feeder(k, SERVE_FEEDER_SEEDS[k]) for k in SERVE_SIZES}
    solvers = {}
    srv = opf.Server(rho=RHO, eps_rel=EPS_REL, eps_abs_pres=EPS_ABS, max_iter=args.max_iter,
                     chunk_iters=args.chunk, polish_chunk_iters=args.polish_chunk)
    mid = {}
    caps = {"13": 1024, "34": 1024, "123": 1024}
    # SM partitions (green contexts): the single-instance workers of the
    # 8500-bus feeder on args.big_sms SMs, the batched models on the rest, so
    # that neither takes the other's SMs
    parts = []
    use_big = weights[SERVE_SIZES.index("8500")] > 0
    if use_big and args.big_sms > 0:
        parts = [opf.SMPartition(-args.big_sms, device=local) if args.batched_partition else None]
        parts += [opf.SMPartition(args.big_sms, device=local) for _ in range(args.big_handles)]
    for j, k in enumerate(SERVE_SIZES):
        if weights[j] == 0:
            continue
        hs = []
        for h in range(args.big_handles if k == "8500" else 1):
            stream = None
            if parts:
                if k == "8500":
                    stream = parts[1 + h].stream
                elif args.batched_partition:
                    stream = parts[0].stream
            sv = opf.Solver.from_feeder(feeders[k], device=local, stream=stream)
            sv.precompute()
            hs.append(sv)
        solvers[k] = hs
        mid[k] = srv.add_model(hs, caps.get(k, 1))
        if k != "8500" and args.serve_k:
            srv.set_model_shape(mid[k], args.serve_k, args.serve_warps)
        if SINGLE_EPS_REL[k] != EPS_REL:
            srv.set_model_tolerance(mid[k], SINGLE_EPS_REL[k], EPS_ABS)   # the large feeder's stopping rule
        srv.set_admission(mid[k], max_wait_s=args.max_wait_s,
                          max_service_s=args.max_service_s if k == "8500" else 0.0)
    rng = np.random.default_rng(SERVE_ARRIVAL_SEED)
    n_total = requests + warm_requests
    gaps = rng.exponential(1.0 / args.rate, size=n_total)
    arrival = np.cumsum(gaps)
    kind = rng.choice(len(SERVE_SIZES), size=n_total, p=weights)
    loads = []
    for r in range(n_total):
        g = synth.load_scenario(feeders[SERVE_SIZES[kind[r]]], SERVE_REQ_SEED0 + r)
        loads.append((g["load_a"], g["load_b"]))
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t0 = time.perf_counter()
    nxt = 0
    done_t, results, refused = {}, {}, set()
    drain_deadline = None
    while True:
        t_pass = time.perf_counter()
        now = t_pass - t0
        while nxt < n_total and arrival[nxt] <= now:
            if not srv.submit(mid[SERVE_SIZES[kind[nxt]]], loads[nxt][0], loads[nxt][1], tag=nxt, refusable=True):
                refused.add(nxt)
            nxt += 1
        srv.step()
        tnow = time.perf_counter() - t0
        for res in srv.poll():
            done_t[res["tag"]] = tnow
            results[res["tag"]] = res
        if nxt == n_total:
            if drain_deadline is None:
                drain_deadline = tnow + drain_s
            if len(results) + len(refused) == n_total or tnow > drain_deadline:
                break
        st = srv.stats()
        if st["running"] == 0 and st["queued"] == 0 and nxt < n_total:
            time.sleep(max(0.0, min(arrival[nxt] - (time.perf_counter() - t0), 0.01)))
        elif time.perf_counter() - t_pass < 1e-3:
            time.sleep(5e-4)            # only worker threads are busy
    elapsed = time.perf_counter() - t0
    clocks = sampler.stop()
    stats = srv.stats()
    model_stats = {k: srv.model_stats(mid[k]) for k in mid}
    measured = range(warm_requests, n_total)
    t_first = arrival[warm_requests]
    cls = {k: {"submitted": 0, "served": 0, "converged": 0, "refused": 0, "shed": 0, "stopped": 0,
               "unfinished": 0, "lat": []} for k in SERVE_SIZES}
    for r in measured:
        c = cls[SERVE_SIZES[kind[r]]]
        c["submitted"] += 1
        if r in refused:
            c["refused"] += 1
        elif r not in results:
            c["unfinished"] += 1               # still queued or running when the window closed
        elif results[r]["status"] == opf.OPF_E_TIMEOUT:
            c["stopped" if results[r]["iters"] > 0 else "shed"] += 1
        else:
            c["served"] += 1
            c["converged"] += int(results[r]["converged"])
            c["lat"].append(1e3 * (done_t[r] - arrival[r]))
    t_last = max((done_t[r] for r in measured if r in done_t), default=elapsed)
    window = max(t_last - t_first, 1e-9)

    def pct(v, q):
        return float(np.percentile(v, q)) if v else None
    per_class = {}
    for k in SERVE_SIZES:
        c = cls[k]
        lat = c.pop("lat")
        per_class[k] = dict(c, p50_ms=pct(lat, 50), p99_ms=pct(lat, 99), solves_per_s=c["converged"] / window)
    all_lat = [1e3 * (done_t[r] - arrival[r]) for r in measured
               if r in results and results[r]["status"] == opf.OPF_OK]
    converged = sum(per_class[k]["converged"] for k in SERVE_SIZES)
    srv.close()
    for hs in solvers.values():
        for sv in hs:
            sv.close()
    for p in parts:
        if p is not None:
            p.close()
    return {"value": converged / window, "p50_ms": pct(all_lat, 50), "p99_ms": pct(all_lat, 99),
            "per_class": per_class, "elapsed_s": elapsed, "window_s": window, "server": stats,
            "models": model_stats, "clocks": clocks, "requests": requests, "warm_requests": warm_requests}


def run_serve(args, rank, world, local):
    import __graft_entry__
    __graft_entry__.build()
    r = serve_measure(args, local, args.requests, args.warm_requests, args.drain_s)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": r["server"]["passes"],
            "warmup": args.warm_requests, "ms_per_step": 1e3 * r["elapsed_s"] / max(r["server"]["passes"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": serve_config(args),
            "latency_ms": {"p50": r["p50_ms"], "p99": r["p99_ms"],
                           "note": "served requests, from the request's arrival time to the pass that retired it"},
            "per_class": r["per_class"], "elapsed_s": r["elapsed_s"], "server": r["server"],
            "models": r["models"], "clocks": r["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch", "single", "serve"])
    ap.add_argument("--requests", type=int, default=4000, help="serve: measured requests")
    ap.add_argument("--warm-requests", type=int, default=200, help="serve: warm-up requests")
    ap.add_argument("--rate", type=float, default=SERVE_RATE, help="serve: mean arrivals per second")
    ap.add_argument("--drain-s", type=float, default=30.0, help="serve: longest drain after the last arrival")
    ap.add_argument("--max-wait-s", type=float, default=2.0,
                    help="serve: admission bound on a request's wait for a slot (predicted at submit, shed after)")
    ap.add_argument("--max-service-s", type=float, default=5.0,
                    help="serve: bound on an 8500-bus request's run time once admitted")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="batch workload: measured requests of the serving sub-record (0: none)")
    ap.add_argument("--no-single-records", dest="single_records", action="store_false",
                    help="batch workload: skip the single-instance sub-records (13/123/8500 buses)")
    ap.add_argument("--big-handles", type=int, default=2, help="serve: 8500-bus worker handles")
    ap.add_argument("--serve-k", type=int, default=2,
                    help="serve: FP32 instances per CTA of the batched models (0: autotuned on a full batch)")
    ap.add_argument("--serve-warps", type=int, default=16, help="serve: warps per CTA of the batched models")
    ap.add_argument("--max-iter", type=int, default=1_000_000, help="serve: iteration cap per request")
    ap.add_argument("--mix", default="0.4,0.3,0.2,0.1", help="serve: weights of the 13/34/123/8500-bus requests")
    ap.add_argument("--big-sms", type=int, default=16, help="serve: SMs of the 8500-bus workers' partition (0: none)")
    ap.add_argument("--batched-partition", action="store_true",
                    help="serve: batched models on a partition of the SMs the 8500-bus workers do not hold "
                         "(default: ordinary streams; measured sevenfold slower passes on the partition)")
    ap.add_argument("--chunk", type=int, default=1000,
                    help="serve: FP32 iterations per pass (and re-centring interval)")
    ap.add_argument("--polish-chunk", type=int, default=0,
                    help="serve: FP64 iterations per pass of slots in the polish (0: the library default)")
    ap.add_argument("--instances", type=int, default=N_SCEN)
    ap.add_argument("--feeder", default="123", choices=sorted(SINGLE_SEEDS, key=int),
                    help="single-instance workload: the feeder (13, 123 and 8500 buses are the single-instance "
                         "configurations)")
    ap.add_argument("--fixed-iters", type=int, default=0,
                    help="single: run exactly this many iterations per step, no stopping test (profiling)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="single-instance workload only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain-fp64", action="store_true",
                    help="batch: skip the plain single-instance FP64 reference solves (profiling runs)")
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
    try:
        if args.workload == "batch":
            return run_batch(args, rank, world, local)
        if args.workload == "serve":
            return run_serve(args, rank, world, local)
        return run_single(args, rank, world, local)
    finally:
        if world > 1:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
