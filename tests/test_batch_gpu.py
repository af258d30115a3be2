"""GPU parity of batched solves (many load scenarios of one feeder) through the C ABI.

* FP64 iterates of every instance after 100 iterations within 1e-10 relative of
  the oracle run on that instance's own model (scenario loads in the rhs);
* FP32 iterations stay within single-precision distance of the oracle;
* mixed-precision solves reach each instance's LP optimum within 1e-6 relative
  with pres <= 1e-4, on small batches and on the full 1024-scenario batch
  (every instance checked against the oracle's LP optimum, computed on a
  pool of host processes).
"""
import numpy as np
import pytest

from oracle import admm as oracle_admm, lindist
from paper_2310_09410_gb300 import opf, synth

pytestmark = pytest.mark.gpu

TOL_ITER = 1e-10
TOL_OBJ = 1e-6
TOL_PRES = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def scenarios(f, seeds):
    return [synth.load_scenario(f, s) for s in seeds]


def load_arrays(fs):
    return (np.stack([g["load_a"] for g in fs]), np.stack([g["load_b"] for g in fs]))


def oracle_iterates(M, iters, rho=100.0):
    return oracle_admm.admm(oracle_admm.Prepared(M), rho=rho, max_iter=iters, check_every=0)


@pytest.mark.parametrize("name,seed,n_scen,k64", [("123", 2001, 6, 4), ("13", 1001, 5, 2), ("34", 5034, 3, 1)])
def test_fp64_batch_iterates_match_oracle(name, seed, n_scen, k64):
    f = synth.preset_feeder(name, seed)
    fs = scenarios(f, [4000 + j for j in range(n_scen)])
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n_scen + 1) as b:            # the last instance keeps the feeder's own loads
            b.set_shape(opf.PREC_FP64, k64)
            lp, lq = load_arrays(fs)
            b.set_loads(0, lp, lq)
            b.step(100)
            for j, g in enumerate(fs + [f]):
                ref = oracle_iterates(lindist.build(g), 100)
                xs, lam = b.locals(j)
                assert rel_err(xs, ref.xs) <= TOL_ITER, j
                assert rel_err(lam, ref.lam) <= TOL_ITER, j
            x, obj = b.solution()
            ref = oracle_iterates(lindist.build(fs[0]), 100)
            assert rel_err(x[0], ref.x) <= TOL_ITER
            assert abs(obj[0] - ref.objective) <= TOL_ITER * max(1.0, abs(ref.objective))


def test_fp64_batch_generic_rank_deficient_rhs():
    g = synth.random_generic(4, max_n=40, n_global=120)
    M = lindist.from_generic(g)
    rng = np.random.default_rng(9)
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        with opf.Batch(s, 3) as b:
            rhs, models = [], []
            for j in range(3):
                subs = []
                for sub in g["subs"]:
                    A = np.asarray(sub["A"], float)
                    bnew = A @ rng.normal(size=A.shape[1])        # consistent by construction
                    subs.append(dict(sub, b=bnew))
                rhs.append(np.concatenate([sb["b"] for sb in subs]))
                models.append(lindist.from_generic(dict(g, subs=subs)))
            b.set_rhs(0, np.stack(rhs))
            b.step(100, rho=3.0)
            for j in range(3):
                ref = oracle_iterates(models[j], 100, rho=3.0)
                xs, lam = b.locals(j)
                assert rel_err(xs, ref.xs) <= TOL_ITER
                assert rel_err(lam, ref.lam) <= TOL_ITER
            # an inconsistent rhs is rejected and named
            bad = rhs[0].copy()
            bad += 1.0
            deficient = any(np.linalg.matrix_rank(np.asarray(sb["A"], float)) < np.asarray(sb["A"]).shape[0]
                            for sb in g["subs"])
            if deficient:
                with pytest.raises(opf.OPFError) as e:
                    b.set_rhs(1, bad[None, :])
                assert e.value.code == opf.OPF_E_INFEASIBLE_LOCAL
    assert M.n == len(g["c"])


@pytest.mark.parametrize("seed", [11, 12])
def test_batch_generic_free_globals(seed):
    """Globals without bounds, with one copy (which the batched engine leaves
    out of its global update: with the shifted cost zero there, rho x is the
    u of the copy's slot) and with several, beside bounded ones, each with a
    cost: FP64 iterates to 1e-10 and FP32 iterates to 1e-4 of the oracle's
    after 100 iterations, on several right-hand sides."""
    g = synth.random_generic(seed, n_global=150, n_sub=14, max_n=30, p_free=0.6)
    copies = np.zeros(len(g["c"]), int)
    for sub in g["subs"]:
        copies[np.asarray(sub["idx"])] += 1
    free = ~np.isfinite(g["lb"]) & ~np.isfinite(g["ub"])
    assert np.any(free & (copies == 1)) and np.any(free & (copies > 1)) and np.any(~free)
    rng = np.random.default_rng(seed)
    subs_j, rhs = [], []
    for j in range(3):
        subs = []
        for sub in g["subs"]:
            A = np.asarray(sub["A"], float)
            subs.append(dict(sub, b=A @ rng.uniform(-0.4, 0.4, A.shape[1])))
        subs_j.append(subs)
        rhs.append(np.concatenate([sb["b"] for sb in subs]))
    refs = [oracle_iterates(lindist.from_generic(dict(g, subs=subs)), 100, rho=3.0) for subs in subs_j]
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        with opf.Batch(s, 3) as b:
            b.set_rhs(0, np.stack(rhs))
            b.step(100, rho=3.0)
            for j in range(3):
                xs, lam = b.locals(j)
                assert rel_err(xs, refs[j].xs) <= TOL_ITER
                assert rel_err(lam, refs[j].lam) <= TOL_ITER
            b.set_rhs(0, np.stack(rhs))
            b.solve(rho=3.0, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP32)
            assert np.all(b.status()["iters"] == 100)
            for j in range(3):
                xs, lam = b.locals(j)
                assert rel_err(xs, refs[j].xs) <= 1e-4
                assert rel_err(lam, refs[j].lam) <= 1e-4


def test_batch_without_global_update_items():
    """One subsystem holding every global, none bounded: every global has one
    copy and no bounds, so the batched engine's global update has no item at
    all (each slot's u is rho x of its global).  FP64 iterates to 1e-10 and
    FP32 iterates to 1e-4 of the oracle's after 100 iterations."""
    g = synth.random_generic(21, n_global=60, n_sub=1, max_n=60, p_free=1.0)
    assert len(g["subs"]) == 1 and not np.any(np.isfinite(g["lb"])) and not np.any(np.isfinite(g["ub"]))
    rng = np.random.default_rng(21)
    subs_j, rhs = [], []
    for j in range(2):
        A = np.asarray(g["subs"][0]["A"], float)
        subs = [dict(g["subs"][0], b=A @ rng.uniform(-0.4, 0.4, A.shape[1]))]
        subs_j.append(subs)
        rhs.append(subs[0]["b"])
    refs = [oracle_iterates(lindist.from_generic(dict(g, subs=subs)), 100, rho=3.0) for subs in subs_j]
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        with opf.Batch(s, 2) as b:
            b.set_rhs(0, np.stack(rhs))
            b.step(100, rho=3.0)
            for j in range(2):
                xs, lam = b.locals(j)
                assert rel_err(xs, refs[j].xs) <= TOL_ITER
                assert rel_err(lam, refs[j].lam) <= TOL_ITER
            b.set_rhs(0, np.stack(rhs))
            b.solve(rho=3.0, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP32)
            for j in range(2):
                xs, lam = b.locals(j)
                assert rel_err(xs, refs[j].xs) <= 1e-4
                assert rel_err(lam, refs[j].lam) <= 1e-4


@pytest.mark.parametrize("k32", [8, 4])
def test_fp32_batch_tracks_oracle(k32):
    f = synth.preset_feeder("123", 2001)
    fs = scenarios(f, [4100, 4101, 4102])
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, 3) as b:
            b.set_shape(opf.PREC_FP32, k32)
            b.set_loads(0, *load_arrays(fs))
            b.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP32)
            st = b.status()
            assert np.all(st["iters"] == 100)
            for j, g in enumerate(fs):
                ref = oracle_iterates(lindist.build(g), 100)
                xs, lam = b.locals(j)
                assert rel_err(xs, ref.xs) <= 1e-4
                assert rel_err(lam, ref.lam) <= 1e-4


@pytest.mark.parametrize("name,seed,n_scen", [("13", 1003, 6), ("123", 2002, 5)])
def test_batch_converged_objective(name, seed, n_scen):
    f = synth.preset_feeder(name, seed)
    fs = scenarios(f, [4200 + j for j in range(n_scen)])
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n_scen) as b:
            b.set_loads(0, *load_arrays(fs))
            ok = b.solve(precision=opf.PREC_MIXED)
            st = b.status()
            _, obj = b.solution()
            assert b.shape(opf.PREC_FP32)["ok"] == 1
            assert len(b.tune_log()) >= 2
    assert ok
    assert np.all(st["converged"])
    assert np.all(st["pres"] <= TOL_PRES)
    for j, g in enumerate(fs):
        obj_star, _ = oracle_admm.lp_optimum(lindist.build(g))
        assert abs(obj[j] - obj_star) <= TOL_OBJ * abs(obj_star), (j, obj[j], obj_star)


@pytest.mark.parametrize("name,seed,n,k,w", [("123", 2001, 24, 8, 16), ("123", 2001, 10, 4, 12),
                                             ("13", 1001, 12, 8, 8), ("34", 5034, 9, 2, 16)])
def test_fp32_engine_tensor_memory_matches_l2_streaming(name, seed, n, k, w):
    """The FP32 engine with lambda and bbar~ held in tensor memory gives
    bit-identical iterates to the same engine shape streaming them from L2
    (the arithmetic is the same; only where the two arrays live differs)."""
    f = synth.preset_feeder(name, seed)
    fs = scenarios(f, [4700 + j for j in range(n)])
    out = {}
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n) as b:
            for tm in (True, False):
                b.set_tmem(tm)
                b.set_shape(opf.PREC_FP32, k, w)
                b.set_loads(0, *load_arrays(fs))
                b.solve(eps_rel=0.0, max_iter=400, check_every=50, precision=opf.PREC_FP32)
                sh = b.shape(opf.PREC_FP32)
                assert sh["tmem"] == (1 if tm else 0) and sh["k_inst"] == k and sh["warps"] == w
                out[tm] = [b.locals(j) for j in range(n)]
                assert np.all(b.status()["iters"] == 400)
    for j in range(n):
        assert np.array_equal(out[True][j][0], out[False][j][0]), j
        assert np.array_equal(out[True][j][1], out[False][j][1]), j


def test_fp32_engine_tensor_memory_freezes_finished_instances():
    """Instances that stop at different test iterations inside one launch:
    each keeps the lambda of its stopping iteration (written from tensor
    memory when it froze), so results equal the L2-streaming engine's."""
    f = synth.preset_feeder("13", 1001)
    fs = scenarios(f, [4800 + j for j in range(16)])
    res = {}
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, len(fs)) as b:
            for tm in (True, False):
                b.set_tmem(tm)
                b.set_shape(opf.PREC_FP32, 8, 16)
                b.set_loads(0, *load_arrays(fs))
                assert b.solve(eps_rel=1e-5, precision=opf.PREC_FP32, recenter_every=4000)
                st = b.status()
                res[tm] = (st["iters"].copy(), [b.locals(j) for j in range(len(fs))])
    assert len(set(res[True][0].tolist())) > 1          # the instances stopped at different iterations
    assert np.array_equal(res[True][0], res[False][0])
    for j in range(len(fs)):
        assert np.array_equal(res[True][1][j][1], res[False][1][j][1]), j


def _lp_optimum_of_scenario(args):
    """Oracle LP optimum of load scenario `seed` of a preset feeder (runs in
    a worker process)."""
    name, fseed, seed = args
    f = synth.preset_feeder(name, fseed)
    return oracle_admm.lp_optimum(lindist.build(synth.load_scenario(f, seed)))[0]


def oracle_lp_optima(name, fseed, seeds):
    """LP optima of many scenarios on a spawn pool (safe after CUDA is up)."""
    import multiprocessing as mp
    import os
    n = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return np.array(pool.map(_lp_optimum_of_scenario, [(name, fseed, sd) for sd in seeds],
                                 chunksize=max(1, len(seeds) // (4 * n))))


def test_full_batch_all_instances_against_oracle():
    """The 1024-scenario batch of the 123-bus feeder as the benchmark runs it;
    every instance's objective is checked against the oracle's LP optimum."""
    f = synth.preset_feeder("123", 2001)
    n = 1024
    seeds = [4000 + j for j in range(n)]
    fs = scenarios(f, seeds)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n) as b:
            b.set_loads(0, *load_arrays(fs))
            ok = b.solve(precision=opf.PREC_MIXED)
            st = b.status()
            _, obj = b.solution()
    assert ok
    assert np.all(st["converged"]) and np.all(st["pres"] <= TOL_PRES)
    obj_star = oracle_lp_optima("123", 2001, seeds)
    rel = np.abs(obj - obj_star) / np.abs(obj_star)
    assert np.all(rel <= TOL_OBJ), (int(np.argmax(rel)), float(rel.max()))


def test_batch_errors():
    f = synth.preset_feeder("13", 1001)
    with opf.Solver.from_feeder(f) as s:
        with pytest.raises(opf.OPFError) as e:
            opf.Batch(s, 2)                                   # not precomputed
        assert e.value.code == opf.OPF_E_STATE
        s.precompute()
        with opf.Batch(s, 2) as b:
            with pytest.raises(opf.OPFError):
                b.solution()                                  # no iteration yet
            with pytest.raises(opf.OPFError) as e:
                b.set_loads(1, np.zeros((2, len(f["load_bus"]), 3)), np.zeros((2, len(f["load_bus"]), 3)))
            assert e.value.code == opf.OPF_E_INVALID         # range past the end
            with pytest.raises(opf.OPFError):
                b.set_shape(opf.PREC_FP32, 3)
    fz = synth.with_zip_delta(synth.preset_feeder("34", 5034), seed=3)
    with opf.Solver.from_feeder(fz) as s:
        s.precompute()
        with opf.Batch(s, 1) as b:
            with pytest.raises(opf.OPFError) as e:
                b.set_loads(0, fz["load_a"][None], fz["load_b"][None])
            assert e.value.code == opf.OPF_E_INVALID
