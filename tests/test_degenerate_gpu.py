"""GPU parity on the degenerate inputs of the method, through the C ABI.

* the smallest feeder (two buses, one line, one load; with and without a
  DER): FP64 iterates after 100 iterations within 1e-10 of the oracle on
  every single-instance engine and in batches of one and of three instances;
* a consensus instance of a single subsystem, where every global has one
  copy and the global update (Eq. closed_1) is the clip of that copy's
  u / rho minus c / rho, on every engine;
* runs of one test interval, and caps between two tests (applied at the
  next test);
* a batch of zero instances is refused.
"""
import numpy as np
import pytest

from oracle import admm as oracle_admm, lindist
from paper_2310_09410_gb300 import opf, synth

pytestmark = pytest.mark.gpu

TOL_ITER = 1e-10
ENGINES = [(opf.ENGINE_GRID, 0), (opf.ENGINE_CTA, 1), (opf.ENGINE_CTA, 2), (opf.ENGINE_WARP, 0),
           (opf.ENGINE_PERSISTENT, 1), (opf.ENGINE_PERSISTENT, 4)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def two_bus(n_der):
    return synth.make_feeder(2, 1, n_der, seed=3 + n_der)


def check(s, ref):
    xs, lam = s.locals()
    x, _ = s.solution()
    assert rel_err(xs, ref.xs) <= TOL_ITER
    assert rel_err(lam, ref.lam) <= TOL_ITER
    assert rel_err(x, ref.x) <= TOL_ITER


@pytest.mark.parametrize("n_der", [0, 1])
@pytest.mark.parametrize("engine,cluster", ENGINES)
def test_two_bus_feeder_every_engine(n_der, engine, cluster):
    f = two_bus(n_der)
    M = lindist.build(f)
    ref = oracle_admm.admm(oracle_admm.Prepared(M), rho=100.0, max_iter=100, check_every=0)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64, engine=engine,
                cluster=cluster)
        assert s.residuals()["iters"] == 100
        check(s, ref)


@pytest.mark.parametrize("n", [1, 3])
def test_two_bus_feeder_batch(n):
    f = two_bus(1)
    fs = [synth.load_scenario(f, 7100 + j) for j in range(n)]
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n) as b:
            b.set_loads(0, np.stack([g["load_a"] for g in fs]), np.stack([g["load_b"] for g in fs]))
            b.step(100)
            got = [b.locals(j) for j in range(n)]
    for j, g in enumerate(fs):
        ref = oracle_admm.admm(oracle_admm.Prepared(lindist.build(g)), rho=100.0, max_iter=100, check_every=0)
        assert rel_err(got[j][0], ref.xs) <= TOL_ITER
        assert rel_err(got[j][1], ref.lam) <= TOL_ITER


@pytest.mark.parametrize("engine,cluster", ENGINES[:5])
def test_single_subsystem_instance(engine, cluster):
    g = synth.random_generic(5, n_global=7, n_sub=1, max_n=7)
    M = lindist.from_generic(g)
    rho = 3.0
    ref = oracle_admm.admm(oracle_admm.Prepared(M), rho=rho, max_iter=100, check_every=0)
    with opf.Solver.from_generic(g["c"], g["lb"], g["ub"], g["subs"]) as s:
        s.precompute()
        s.solve(rho=rho, eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP64, engine=engine,
                cluster=cluster)
        check(s, ref)


@pytest.mark.parametrize("engine", [opf.ENGINE_GRID, opf.ENGINE_CTA, opf.ENGINE_WARP, opf.ENGINE_PERSISTENT])
def test_short_runs_and_cap_between_tests(engine):
    """One test interval (2 iterations), and a cap between two tests: the
    cap is applied at the tests, so max_iter = 1 and 3 run 2 and 4
    iterations, on every engine, each matching the oracle run as long."""
    f = synth.preset_feeder("13", 1001)
    M = lindist.build(f)
    for cap, iters in ((1, 2), (2, 2), (3, 4)):
        ref = oracle_admm.admm(oracle_admm.Prepared(M), rho=100.0, max_iter=iters, check_every=0)
        with opf.Solver.from_feeder(f) as s:
            s.precompute()
            ok = s.solve(eps_rel=0.0, max_iter=cap, check_every=2, precision=opf.PREC_FP64, engine=engine)
            assert not ok
            assert s.residuals()["iters"] == iters
            check(s, ref)


def test_empty_batch_refused():
    f = two_bus(0)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with pytest.raises(opf.OPFError) as e:
            opf.Batch(s, 0)
        assert e.value.code == opf.OPF_E_INVALID
