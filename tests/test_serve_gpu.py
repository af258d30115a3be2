"""GPU tests of the request server (continuous batching) through the C ABI.

* a request gives the same result (iterations, objective, x bit for bit)
  alone and when admitted later among requests of other feeders and
  scenarios;
* served results reach each request's LP optimum within 1e-6 relative;
* admission is bounded by the device-memory budget;
* models too large for the batched engine are served by worker threads;
* a model's admission policy serves, refuses at submit or sheds every
  request with a counted status (none is left pending).
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


def test_flooded_worker_model_serves_or_refuses_every_request():
    """A model served by worker threads (ZIP loads: a factorization per
    request) with a bounded queue: every request of a burst is either served
    or refused at submit with a status, and none is left pending."""
    fz = synth.with_zip_delta(synth.preset_feeder("34", 5034), seed=11)
    h = solver(fz)
    n = 10
    with opf.Server() as srv:
        m = srv.add_model([h], capacity=4)
        srv.set_admission(m, max_queue=2)
        accepted = []
        for r in range(n):
            g = synth.load_scenario(fz, 6700 + r)
            if srv.submit(m, g["load_a"], g["load_b"], tag=r, refusable=True):
                accepted.append(r)
        assert 2 <= len(accepted) < n
        got = drain(srv, accepted)
        st = srv.model_stats(m)
    assert st["submitted"] == n
    assert st["refused"] == n - len(accepted)
    assert st["served"] == len(accepted) and st["shed"] == 0
    assert st["queued"] == 0 and st["running"] == 0
    for r in accepted:
        assert got[r]["status"] == opf.OPF_OK and got[r]["converged"]
    h.close()


def test_waiting_requests_are_shed_then_refused_by_predicted_wait():
    """max_wait_s: queued requests that wait longer are shed with
    OPF_E_TIMEOUT; once the model has a measured service time, a request
    whose predicted wait exceeds the bound is refused at submit."""
    fz = synth.with_zip_delta(synth.preset_feeder("123", 5123), seed=12)
    h = solver(fz)
    scen = [synth.load_scenario(fz, 6800 + r) for r in range(8)]
    with opf.Server() as srv:
        m = srv.add_model([h], capacity=4)
        srv.set_admission(m, max_wait_s=0.02)
        assert srv.submit(m, scen[0]["load_a"], scen[0]["load_b"], tag=0, refusable=True)
        srv.step()                                          # the worker takes request 0
        for r in range(1, 4):                               # no service time yet: queued
            assert srv.submit(m, scen[r]["load_a"], scen[r]["load_b"], tag=r, refusable=True)
        got = drain(srv, list(range(4)))
        st = srv.model_stats(m)
        assert got[0]["status"] == opf.OPF_OK and got[0]["converged"]
        shed = [r for r in range(1, 4) if got[r]["status"] == opf.OPF_E_TIMEOUT]
        assert shed, got                                    # one worker, 20 ms bound, solves take longer
        for r in shed:
            assert not got[r]["converged"] and np.isnan(got[r]["objective"])
        assert st["service_s"] > 0.02
        # a free worker admits one request; the next would wait a service time
        assert srv.submit(m, scen[4]["load_a"], scen[4]["load_b"], tag=4, refusable=True)
        assert not srv.submit(m, scen[5]["load_a"], scen[5]["load_b"], tag=5, refusable=True)
        got.update(drain(srv, [4]))
        st = srv.model_stats(m)
    assert st["submitted"] == 6 and st["refused"] == 1
    assert st["served"] + st["shed"] + st["refused"] == st["submitted"]
    assert st["queued"] == 0 and st["running"] == 0
    assert got[4]["status"] == opf.OPF_OK
    h.close()


def test_service_bound_stops_running_requests_with_a_status():
    """max_service_s: a worker's solve stops at its next chunk and a batched
    slot is retired at the end of a pass once the bound has passed; both are
    reported with OPF_E_TIMEOUT and counted as stopped."""
    fz = synth.with_zip_delta(synth.preset_feeder("123", 5123), seed=13)
    f13 = synth.preset_feeder("13", 5013)
    hz, h13 = solver(fz), solver(f13)
    with opf.Server() as srv:
        mz = srv.add_model([hz], capacity=4)
        m13 = srv.add_model([h13], capacity=8)
        srv.set_admission(mz, max_service_s=1e-3)
        srv.set_admission(m13, max_service_s=1e-6)
        g = synth.load_scenario(fz, 6900)
        srv.submit(mz, g["load_a"], g["load_b"], tag=0)
        for r in range(3):
            g = synth.load_scenario(f13, 6910 + r)
            srv.submit(m13, g["load_a"], g["load_b"], tag=1 + r)
        got = drain(srv, [0, 1, 2, 3])
        stz, st13 = srv.model_stats(mz), srv.model_stats(m13)
    for r in range(4):
        assert got[r]["status"] == opf.OPF_E_TIMEOUT and not got[r]["converged"]
        assert np.isnan(got[r]["objective"])
    assert stz["stopped"] == 1 and stz["served"] == 1 and stz["converged"] == 0
    assert st13["stopped"] == 3 and st13["served"] == 3
    for st in (stz, st13):
        assert st["queued"] == 0 and st["running"] == 0
    hz.close()
    h13.close()


def test_no_history_wait_predicted_from_running_requests():
    """Before any request of a model has finished, the predicted wait uses
    the time the running request has run so far (a lower bound on its
    service time): a request that would have to wait longer than max_wait_s
    is refused at submit instead of queued and shed later."""
    import time
    fz = synth.with_zip_delta(synth.preset_feeder("123", 5123), seed=14)
    h = solver(fz)
    with opf.Server() as srv:
        m = srv.add_model([h], capacity=1)
        srv.set_model_tolerance(m, 1e-15, 1e-15)       # runs until stopped
        srv.set_admission(m, max_wait_s=0.1, max_service_s=0.6)
        g = synth.load_scenario(fz, 7000)
        assert srv.submit(m, g["load_a"], g["load_b"], tag=0, refusable=True)
        srv.step()                                     # the worker takes request 0
        time.sleep(0.2)
        g = synth.load_scenario(fz, 7001)
        assert not srv.submit(m, g["load_a"], g["load_b"], tag=1, refusable=True)
        got = drain(srv, [0])
        st = srv.model_stats(m)
    assert got[0]["status"] == opf.OPF_E_TIMEOUT and got[0]["iters"] > 0
    assert st["submitted"] == 2 and st["refused"] == 1 and st["stopped"] == 1 and st["shed"] == 0
    assert st["queued"] == 0 and st["running"] == 0
    h.close()


def test_model_shape_fixed_for_latency():
    """A batched model served with a fixed small shape (2 instances per CTA):
    its requests converge to the LP optimum and a request's result is the
    same alone and among others; worker models and bad shapes are refused."""
    f = synth.preset_feeder("34", 5034)
    h = solver(f)
    fz = synth.with_zip_delta(synth.preset_feeder("34", 5034), seed=15)
    hz = solver(fz)
    target = synth.load_scenario(f, 7100)
    with opf.Server() as srv:
        m = srv.add_model([h], capacity=64)
        mz = srv.add_model([hz], capacity=2)
        srv.set_model_shape(m, 2, 16)
        for bad in ((3, 16), (2, 17)):
            with pytest.raises(opf.OPFError) as e:
                srv.set_model_shape(m, *bad)
            assert e.value.code == opf.OPF_E_INVALID
        srv.set_model_shape(m, 2, 16)
        with pytest.raises(opf.OPFError) as e:
            srv.set_model_shape(mz, 2, 16)
        assert e.value.code == opf.OPF_E_INVALID
        srv.submit(m, target["load_a"], target["load_b"], tag=0)
        alone = drain(srv, [0])[0]
        for r in range(1, 13):
            g = synth.load_scenario(f, 7100 + r)
            srv.submit(m, g["load_a"], g["load_b"], tag=r)
        srv.step()
        srv.submit(m, target["load_a"], target["load_b"], tag=99)
        got = drain(srv, list(range(1, 13)) + [99])
    assert alone["converged"] and got[99]["converged"]
    assert alone["iters"] == got[99]["iters"] and alone["objective"] == got[99]["objective"]
    star, _ = oracle_admm.lp_optimum(lindist.build(target))
    assert abs(alone["objective"] - star) <= TOL_OBJ * abs(star)
    for r in range(1, 13):
        assert got[r]["converged"]
    h.close()
    hz.close()
