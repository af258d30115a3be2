"""bench.py's JSON line, checked on the CPU through the reference arm (the
oracle timed on the host cores) and the host-side helpers of the GPU arm."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e")


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "single",
                          "--feeder", "13", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for k in KEYS:
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_fp64_engine_rule_and_launch_counts():
    """The launch counts bench.py claims follow the library's automatic FP64
    engine: the warp engine (one launch per solve) up to 64 subsystems of at
    most 64 slots, else the persistent engine (one launch per 20000
    iterations)."""
    small = {"n_sub": 18, "max_ns": 36}
    large = {"n_sub": 188, "max_ns": 51}
    assert bench.warp_engine_fp64(small) and not bench.warp_engine_fp64(large)
    assert not bench.warp_engine_fp64({"n_sub": 12, "max_ns": 94})
    st = {"main_iters": 3150, "polish_iters": 0}
    # precompute (3) + objective read (1) + u (1) + the engine
    assert bench.count_launches_single(st, "fp64", warp64=True) == 3 + 1 + 1 + 1
    st = {"main_iters": 26000, "polish_iters": 0}
    assert bench.count_launches_single(st, "fp64", persistent=True) == 3 + 1 + 1 + 2


def test_oracle_error_of_the_bench_line():
    """The per-result error the bench line reports: objectives of oracle
    solves give errors at the solver's accuracy, a planted offset shows up,
    and pres recomputed from x and x_s matches the recorded one."""
    import numpy as np
    from oracle import admm as oracle_admm, lindist
    from paper_2310_09410_gb300 import synth
    f = synth.preset_feeder("13", 1001)
    fs = [synth.load_scenario(f, 4000 + j) for j in range(3)]
    res = [oracle_admm.admm(oracle_admm.Prepared(lindist.build(g)), rho=100.0, eps_rel=1e-8, eps_abs_pres=1e-4,
                            max_iter=200_000, check_every=50) for g in fs]
    objs = np.array([r.objective for r in res])
    pres = np.array([r.pres for r in res])
    x = np.stack([r.x for r in res])
    out = bench.oracle_error(fs, objs, pres, x=x, locals_of=lambda j: (res[j].xs, res[j].lam), sample=3)
    assert out["instances"] == 3 and out["pres_host_sample"] == 3
    assert out["max_obj_rel"] < 1e-6
    assert out["pres_host_vs_gpu_max_rel_diff"] < 1e-9
    bad = bench.oracle_error(fs, objs * (1 + 1e-3), pres)
    assert 0.9e-3 < bad["max_obj_rel"] < 1.1e-3


def test_issue_roofline_of_the_batched_engine():
    """The issue figure: warp instructions per SM-cycle of the engine's grid
    against 4; one launch of the captured kernel (4000 iterations x 1024
    instances, 16.80 G warp instructions, 25.42 ms single-pass at 2070 MHz on
    128 SMs) gives 2.49 per cycle; other engine shapes get none."""
    shape = {"k_inst": 8, "warps": 16, "tmem": 1, "ctas": 128}
    r = bench.issue_roofline(shape, 4000 * 1024, 25.42, 2070.0)
    assert abs(r["achieved_ipc_per_sm"] - 16.7984e9 / (25.42e-3 * 2070e6 * 128)) < 1e-9
    assert 0.6 < r["frac"] < 0.65 and r["peak_ipc_per_sm"] == 4.0 and r["sms"] == 128
    assert bench.issue_roofline(dict(shape, k_inst=4), 2000 * 1024, 17.59, 2070.0) is None
    assert bench.issue_roofline(shape, 2000 * 1024, 0.0, 2070.0) is None
