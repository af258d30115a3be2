"""GPU parity: the CUDA path against the CPU oracle through the C ABI.

* FP64 iterates (x, x_s, lambda) after 100 iterations within 1e-10 relative
  (whole-grid, cluster, warp and persistent grid engines), on synthetic feeders of every size and on random
  consensus instances (rank-deficient blocks, blocks wider than 64);
  also with non-zero shunts and off-nominal taps on every bus and line;
* converged solves (FP64 and mixed precision) reach the LP optimum of the
  oracle within 1e-6 relative with pres <= 1e-4.
"""
import numpy as np
import pytest

from oracle import admm as oracle_admm, lindist
from paper_2310_09410_gb300 import opf, synth

pytestmark = pytest.mark.gpu

TOL_ITER = 1e-10   # relative, FP64 iterates over the first 100 iterations
TOL_OBJ = 1e-6     # relative objective at convergence
TOL_PRES = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def oracle_iterates(M, iters, rho=100.0):
    P = oracle_admm.Prepared(M)
    return oracle_admm.admm(P, rho=rho, max_iter=iters, check_every=0)


FEEDERS = [("13", 1001), ("13", 1002), ("34", 5034), ("123", 2001), ("8500", 3001)]


@pytest.mark.parametrize("name,seed", FEEDERS)
def test_fp64_iterates_match_oracle(name, seed):
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    ref = oracle_iterates(M, 100)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.step(100)
        xs, lam = s.locals()
        x, obj = s.solution()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER
    assert abs(obj - ref.objective) <= TOL_ITER * max(1.0, abs(ref.objective))


@pytest.mark.parametrize("name,seed,cluster", [("13", 1001, 1), ("13", 1001, 16), ("34", 5034, 4),
                                               ("123", 2001, 8), ("123", 2001, 16)])
def test_cluster_engine_fp64_matches_oracle(name, seed, cluster):
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    ref = oracle_iterates(M, 100)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64, engine=opf.ENGINE_CTA,
                cluster=cluster)
        xs, lam = s.locals()
        x, _ = s.solution()
        assert s.residuals()["iters"] == 100
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER


@pytest.mark.parametrize("name,seed,ctas", [("13", 1001, 1), ("13", 1001, 32), ("34", 5034, 5),
                                            ("123", 2001, 3), ("123", 2001, 40), ("123", 2001, 0),
                                            ("8500", 3001, 0), ("8500", 3001, 152)])
def test_persistent_engine_fp64_matches_oracle(name, seed, ctas):
    """The persistent grid engine (one cooperative launch, grid barrier per
    iteration) with 1 CTA, more CTAs than subsystems, and automatic / fixed
    grids on the large feeder: FP64 iterates match the oracle."""
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    ref = oracle_iterates(M, 100)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64,
                engine=opf.ENGINE_PERSISTENT, cluster=ctas)
        xs, lam = s.locals()
        x, obj = s.solution()
        assert s.residuals()["iters"] == 100
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER
    assert abs(obj - ref.objective) <= TOL_ITER * max(1.0, abs(ref.objective))


@pytest.mark.parametrize("name,seed,ctas", [("13", 1001, 0), ("13", 1002, 0), ("13", 1002, 2), ("13", 1001, 16),
                                            ("34", 5034, 0), ("34", 5034, 9), ("123", 2001, 0)])
def test_warp_engine_fp64_matches_oracle(name, seed, ctas):
    """The FP64 warp engine (one cluster of 2 to 16 CTAs, a warp per
    subsystem or two for the largest ones, factors in shared memory,
    lane-group splits of the mat-vecs of small blocks; blocks of up to 51
    slots here, so every branch runs): FP64 iterates match the oracle."""
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    ref = oracle_iterates(M, 100)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64, engine=opf.ENGINE_WARP,
                cluster=ctas)
        xs, lam = s.locals()
        x, obj = s.solution()
        assert s.residuals()["iters"] == 100
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER
    assert abs(obj - ref.objective) <= TOL_ITER * max(1.0, abs(ref.objective))


@pytest.mark.parametrize("engine", [opf.ENGINE_GRID, opf.ENGINE_CLUSTER, opf.ENGINE_WARP, opf.ENGINE_PERSISTENT])
@pytest.mark.parametrize("name,seed", [("13", 1002), ("34", 5034), ("123", 2001)])
def test_fp32_engines_track_oracle(name, seed, engine):
    """FP32 iterations without re-centring stay within single-precision
    distance of the FP64 oracle over 100 iterations, on every engine."""
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    ref = oracle_iterates(M, 100)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP32, engine=engine)
        xs, lam = s.locals()
        assert s.residuals()["iters"] == 100
    assert rel_err(xs, ref.xs) <= 1e-4
    assert rel_err(lam, ref.lam) <= 1e-4


def generic_model(seed, **kw):
    g = synth.random_generic(seed, **kw)
    return g, lindist.from_generic(g)


@pytest.mark.parametrize("seed,kw", [(1, {}), (7, {}), (4, {"max_n": 40, "n_global": 120}),
                                     (9, {"max_n": 100, "n_global": 160, "n_sub": 5}),
                                     (11, {"p_free": 0.3})])
def test_generic_iterates_match_oracle(seed, kw):
    g, M = generic_model(seed, **kw)
    rho = 3.0
    ref = oracle_iterates(M, 100, rho=rho)
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        s.step(100, rho=rho)
        xs, lam = s.locals()
        x, _ = s.solution()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER


@pytest.mark.parametrize("seed,kw,ctas", [(1, {}, 2), (4, {"max_n": 40, "n_global": 120}, 3),
                                          (11, {"p_free": 0.3}, 5)])
def test_generic_persistent_engine_matches_oracle(seed, kw, ctas):
    """Rank-deficient blocks, free variables and wide blocks on the
    persistent grid engine (a few CTAs, so globals span CTAs)."""
    g, M = generic_model(seed, **kw)
    rho = 3.0
    ref = oracle_iterates(M, 100, rho=rho)
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        s.solve(rho=rho, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64,
                engine=opf.ENGINE_PERSISTENT, cluster=ctas)
        xs, lam = s.locals()
        x, _ = s.solution()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER


@pytest.mark.parametrize("seed,kw", [(1, {}), (4, {"max_n": 40, "n_global": 120}), (11, {"p_free": 0.3})])
def test_generic_warp_engine_fp64_matches_oracle(seed, kw):
    """Rank-deficient blocks and free variables on the FP64 warp engine."""
    g, M = generic_model(seed, **kw)
    rho = 3.0
    ref = oracle_iterates(M, 100, rho=rho)
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        s.solve(rho=rho, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64,
                engine=opf.ENGINE_WARP)
        xs, lam = s.locals()
        x, _ = s.solution()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER


def test_warp_engine_cta_count_limits():
    """engine 3 takes 1 to 16 CTAs holding at most 12 subsystems each: 17 is
    invalid, one CTA cannot hold the 188 subsystems of the 123-bus feeder."""
    f = synth.preset_feeder("123", 2001)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        for prec in (opf.PREC_FP64, opf.PREC_FP32):
            with pytest.raises(opf.OPFError) as e:
                s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=prec, engine=opf.ENGINE_WARP, cluster=17)
            assert e.value.code == opf.OPF_E_INVALID
            with pytest.raises(opf.OPFError) as e:
                s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=prec, engine=opf.ENGINE_WARP, cluster=1)
            assert e.value.code == opf.OPF_E_CAPACITY
        s.reset()
        s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64, engine=opf.ENGINE_WARP, cluster=16)
        assert s.residuals()["iters"] == 100


def test_warp_engine_refuses_wide_blocks():
    """A block of 94 slots does not fit a warp: the FP64 warp engine refuses
    with OPF_E_CAPACITY, and the automatic choice (the persistent grid engine)
    iterates to oracle parity."""
    g, M = generic_model(9, max_n=100, n_global=160, n_sub=5)
    rho = 3.0
    ref = oracle_iterates(M, 100, rho=rho)
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        with pytest.raises(opf.OPFError) as e:
            s.solve(rho=rho, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64,
                    engine=opf.ENGINE_WARP)
        assert e.value.code == opf.OPF_E_CAPACITY
        s.reset()
        s.solve(rho=rho, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64)
        assert s.residuals()["iters"] == 100
        xs, lam = s.locals()
        x, _ = s.solution()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER


def largest_subsystem_instance(seed=17, n=300):
    """A consensus instance whose first subsystem has OPF_MAX_NS = 256 slots
    (rank 120), the others small and overlapping it."""
    rng = np.random.default_rng(seed)
    lb, ub = rng.uniform(-2, 0, n), rng.uniform(0.5, 2, n)
    c, xf = rng.uniform(-1, 1, n), rng.uniform(-0.4, 0.4, n)
    subs = []
    idx = np.arange(256, dtype=np.int32)
    A = rng.normal(size=(120, 256))
    subs.append({"idx": idx, "A": A, "b": A @ xf[idx]})
    for start in range(230, n, 15):
        idx = np.arange(start, min(start + 20, n), dtype=np.int32)
        A = rng.normal(size=(max(1, len(idx) // 3), len(idx)))
        subs.append({"idx": idx, "A": A, "b": A @ xf[idx]})
    return {"c": c, "lb": lb, "ub": ub, "subs": subs}


def test_largest_subsystem_matches_oracle():
    """OPF_MAX_NS slots in one subsystem: FP64 iterates on the whole-grid
    engine match the oracle, a mixed solve reaches the LP optimum, and the
    persistent engine, whose CTA cannot hold that factor in FP64, refuses
    with OPF_E_CAPACITY."""
    g = largest_subsystem_instance()
    assert max(len(s["idx"]) for s in g["subs"]) == 256
    M = lindist.from_generic(g)
    rho = 3.0
    ref = oracle_iterates(M, 100, rho=rho)
    obj_star, _ = oracle_admm.lp_optimum(M)
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        s.step(100, rho=rho)
        xs, lam = s.locals()
        x, _ = s.solution()
        with pytest.raises(opf.OPFError) as e:
            s.solve(rho=rho, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64,
                    engine=opf.ENGINE_PERSISTENT)
        assert e.value.code == opf.OPF_E_CAPACITY
        s.reset()
        assert s.solve(rho=rho, precision=opf.PREC_MIXED, max_iter=2_000_000)
        _, obj = s.solution()
        r = s.residuals()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER
    assert r["pres"] <= TOL_PRES
    assert abs(obj - obj_star) <= TOL_OBJ * max(1.0, abs(obj_star)), (obj, obj_star, r)


def test_zip_delta_loads_match_oracle():
    f = synth.with_zip_delta(synth.preset_feeder("34", 5034), seed=3)
    assert f["load_delta"].sum() > 0
    M = lindist.build(f)
    ref = oracle_iterates(M, 100)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.step(100)
        xs, lam = s.locals()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER


@pytest.mark.parametrize("name,seed,engine", [("34", 5034, opf.ENGINE_AUTO), ("123", 2001, opf.ENGINE_AUTO),
                                              ("123", 2001, opf.ENGINE_GRID), ("13", 1001, opf.ENGINE_PERSISTENT)])
def test_shunts_and_taps_match_oracle(name, seed, engine):
    """Non-zero g^sh, b^sh (Eq. balance_eqns), g^s, b^s at both line ends and
    taps tau != 1 (Eq. power_flow_eqns) on every bus and line: the library's
    own LP rows give the oracle's FP64 iterates over 100 iterations."""
    f = synth.with_shunts_and_taps(synth.preset_feeder(name, seed), seed=77)
    M = lindist.build(f)
    ref = oracle_iterates(M, 100)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64, engine=engine)
        xs, lam = s.locals()
        x, obj = s.solution()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER
    assert abs(obj - ref.objective) <= TOL_ITER * max(1.0, abs(ref.objective))


@pytest.mark.parametrize("precision,engine", [(opf.PREC_FP64, opf.ENGINE_AUTO), (opf.PREC_MIXED, opf.ENGINE_AUTO),
                                              (opf.PREC_FP64, opf.ENGINE_GRID), (opf.PREC_MIXED, opf.ENGINE_GRID),
                                              (opf.PREC_FP64, opf.ENGINE_WARP), (opf.PREC_MIXED, opf.ENGINE_WARP),
                                              (opf.PREC_FP64, opf.ENGINE_PERSISTENT),
                                              (opf.PREC_MIXED, opf.ENGINE_PERSISTENT)])
@pytest.mark.parametrize("name,seed", [("13", 1003), ("123", 2002)])
def test_converged_objective(name, seed, precision, engine):
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    obj_star, _ = oracle_admm.lp_optimum(M)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        ok = s.solve(precision=precision, engine=engine)
        _, obj = s.solution()
        r = s.residuals()
    assert ok
    assert r["pres"] <= TOL_PRES
    assert abs(obj - obj_star) <= TOL_OBJ * abs(obj_star), (obj, obj_star, r)


@pytest.mark.parametrize("name,seed", [("13", 1001), ("34", 5034), ("123", 2001)])
def test_fp32_reaches_paper_tolerance_in_fp64_iterations(name, seed):
    """Sec. V-C / Table V: with the paper's default eps_rel = 1e-3 (the
    Sec. III-C test alone, no absolute gate) FP32 iterations stop at the same
    or nearly the same iteration as FP64 ones (tested every 2 iterations)."""
    f = synth.preset_feeder(name, seed)
    its = {}
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        for prec in (opf.PREC_FP64, opf.PREC_FP32):
            s.reset()
            assert s.solve(eps_rel=1e-3, eps_abs_pres=1e30, max_iter=200_000, check_every=2, precision=prec)
            its[prec] = s.residuals()["iters"]
    it64, it32 = its[opf.PREC_FP64], its[opf.PREC_FP32]
    assert abs(it32 - it64) <= max(4, 0.02 * it64), its


def test_step_then_getters_and_errors():
    f = synth.preset_feeder("13", 1001)
    with opf.Solver.from_feeder(f) as s:
        with pytest.raises(opf.OPFError) as e:
            s.solve()
        assert e.value.code == opf.OPF_E_STATE
        s.precompute()
        s.step(0)
        with pytest.raises(opf.OPFError):
            s.solution()                       # no iteration yet
        s.step(3)                              # odd count
        xs, lam = s.locals()
        s.step(2)
        xs5, lam5 = s.locals()
        s.set_locals(xs, lam)                  # checkpoint restore
        s.step(2)
        xs5b, lam5b = s.locals()
        assert np.array_equal(xs5, xs5b) and np.array_equal(lam5, lam5b)
        ok = s.solve(max_iter=100)
        assert not ok                          # iteration cap, results readable
        x, obj = s.solution()
        assert np.all(np.isfinite(x))


def test_inconsistent_local_system():
    subs = [{"idx": np.array([0, 1]), "A": np.array([[1.0, 1.0], [2.0, 2.0]]), "b": np.array([1.0, 3.0])},
            {"idx": np.array([1, 2]), "A": np.array([[1.0, -1.0]]), "b": np.array([0.0])}]
    with opf.Solver.from_generic(np.zeros(3), -np.ones(3), np.ones(3), subs) as s:
        with pytest.raises(opf.OPFError) as e:
            s.precompute()
        assert e.value.code == opf.OPF_E_INFEASIBLE_LOCAL
