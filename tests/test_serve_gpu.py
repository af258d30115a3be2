"""GPU tests of the request server (continuous batching) through the C ABI.

* a request gives the same result (iterations, objective, x bit for bit)
  alone and when admitted later among requests of other feeders and
  scenarios;
* served results reach each request's LP optimum within 1e-6 relative;
* admission is bounded by the device-memory budget;
* models too large for the batched engine are served by worker threads.
"""
import numpy as np
import pytest

from oracle import admm as oracle_admm, lindist
from paper_2310_09410_gb300 import opf, synth

pytestmark = pytest.mark.gpu

TOL_OBJ = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def solver(f):
    s = opf.Solver.from_feeder(f)
    s.precompute()
    return s


def drain(srv, want, max_passes=2000, max_seconds=300.0):
    import time
    got = {}
    t0 = time.monotonic()
    for _ in range(max_passes):
        srv.step()
        for r in srv.poll():
            got[r["tag"]] = r
        if all(t in got for t in want):
            return got
        if time.monotonic() - t0 > max_seconds:
            break
        if srv.stats()["running"]:
            time.sleep(0.0005)          # worker threads of single-instance models run meanwhile
    raise AssertionError("requests did not finish")


def test_result_identical_alone_and_in_mix():
    f13, f123 = synth.preset_feeder("13", 5013), synth.preset_feeder("123", 5123)
    s13, s123 = solver(f13), solver(f123)
    target = synth.load_scenario(f123, 6000)
    with opf.Server(keep_solutions=True) as srv:
        m13 = srv.add_model([s13], capacity=24)
        m123 = srv.add_model([s123], capacity=24)
        srv.submit(m123, target["load_a"], target["load_b"], tag=1)
        alone = drain(srv, [1])[1]
        x_alone = srv.take_solution(1, m123)
        # a mix: other requests of both feeders, the target admitted two passes later
        tag = 100
        for r in range(12):
            g = synth.load_scenario(f13, 6100 + r)
            srv.submit(m13, g["load_a"], g["load_b"], tag=tag)
            tag += 1
            g = synth.load_scenario(f123, 6200 + r)
            srv.submit(m123, g["load_a"], g["load_b"], tag=tag)
            tag += 1
        srv.step()
        srv.step()
        srv.submit(m123, target["load_a"], target["load_b"], tag=2)
        for r in range(6):
            g = synth.load_scenario(f123, 6300 + r)
            srv.submit(m123, g["load_a"], g["load_b"], tag=tag)
            tag += 1
        got = drain(srv, [2] + list(range(100, tag)))
        mixed = got[2]
        x_mixed = srv.take_solution(2, m123)
        assert srv.stats()["running"] == 0
    assert alone["converged"] and mixed["converged"]
    assert alone["iters"] == mixed["iters"]
    assert alone["objective"] == mixed["objective"]
    assert np.array_equal(x_alone, x_mixed)
    s13.close()
    s123.close()


def test_served_objectives_match_lp_optimum():
    f34 = synth.preset_feeder("34", 5034)
    s34 = solver(f34)
    scen = [synth.load_scenario(f34, 6400 + r) for r in range(5)]
    with opf.Server() as srv:
        m = srv.add_model([s34], capacity=8)
        for r, g in enumerate(scen):
            srv.submit(m, g["load_a"], g["load_b"], tag=r)
        got = drain(srv, list(range(len(scen))))
    for r, g in enumerate(scen):
        obj_star, _ = oracle_admm.lp_optimum(lindist.build(g))
        assert got[r]["converged"]
        assert abs(got[r]["objective"] - obj_star) <= TOL_OBJ * abs(obj_star), (r, got[r], obj_star)
    s34.close()


def test_memory_budget_bounds_slots():
    f13 = synth.preset_feeder("13", 5013)
    s13 = solver(f13)
    with opf.Server(mem_budget=2_000_000) as srv:
        srv.add_model([s13], capacity=100_000)
        st = srv.stats()
        assert 1 <= st["slots"] < 100_000
        assert st["mem_bytes"] <= 2_000_000
    with opf.Server(mem_budget=1000) as srv:
        with pytest.raises(opf.OPFError) as e:
            srv.add_model([s13], capacity=4)
        assert e.value.code == opf.OPF_E_CAPACITY
    s13.close()


def test_large_model_served_by_workers():
    f = synth.preset_feeder("8500", 5850)
    handles = [solver(f), solver(f)]
    with opf.Server(max_iter=2000) as srv:
        m = srv.add_model(handles, capacity=64)
        srv.set_model_tolerance(m, 2e-9, 1e-4)           # the large feeder's stopping rule
        assert srv.stats()["slots"] == 2                 # one request per handle
        for r in range(3):
            g = synth.load_scenario(f, 6500 + r)
            srv.submit(m, g["load_a"], g["load_b"], tag=r)
        got = drain(srv, [0, 1, 2], max_passes=100000)
    for r in range(3):
        assert got[r]["iters"] >= 2000 or got[r]["converged"]
        assert np.isfinite(got[r]["objective"])
    for h in handles:
        h.close()


def test_model_tolerance_applies_to_its_requests():
    f13 = synth.preset_feeder("13", 5013)
    scen = [synth.load_scenario(f13, 6600 + r) for r in range(3)]
    iters = {}
    for eps in (1e-8, 1e-5):
        s13 = solver(f13)
        with opf.Server() as srv:
            m = srv.add_model([s13], capacity=8)
            if eps != 1e-8:
                srv.set_model_tolerance(m, eps, 1e-4)
            for r, g in enumerate(scen):
                srv.submit(m, g["load_a"], g["load_b"], tag=r)
            got = drain(srv, list(range(len(scen))))
        iters[eps] = [got[r]["iters"] for r in range(len(scen))]
        assert all(got[r]["converged"] for r in range(len(scen)))
        s13.close()
    assert all(a < b for a, b in zip(iters[1e-5], iters[1e-8])), iters
