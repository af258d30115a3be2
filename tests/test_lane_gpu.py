"""GPU tests of the lane engine (FP32 batches, one instance per lane, tiles of
128 instances on clusters of CTAs that split the subsystems).

* FP32 iterates after 100 iterations stay within single-precision distance
  (1e-4 relative) of the oracle run on each instance's own model, on the 13-,
  34- and 123-bus feeders (plans of several parts, with globals whose copies
  lie in different parts), with 1 to 4 warps per lane quadrant;
* mixed-precision solves reach each instance's LP optimum within 1e-6 with
  pres <= 1e-4;
* an instance gives bit-identical results and stopping iterations alone and
  in a batch of 130 (two tiles, the second partly empty, instances stopping
  at different test iterations: the freeze of finished lanes);
* a model that needs more parts than a cluster has CTAs is refused.
"""
import numpy as np
import pytest

from oracle import admm as oracle_admm, lindist
from paper_2310_09410_gb300 import opf, synth

pytestmark = pytest.mark.gpu

LANE = 128


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


@pytest.mark.parametrize("name,seed,n,warps", [("13", 1001, 3, 16), ("34", 5034, 4, 8), ("123", 2001, 5, 16),
                                               ("123", 2001, 3, 4)])
def test_lane_fp32_tracks_oracle(name, seed, n, warps):
    f = synth.preset_feeder(name, seed)
    fs = scenarios(f, [4100 + j for j in range(n)])
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n) as b:
            b.set_shape(opf.PREC_FP32, LANE, warps)
            b.set_loads(0, *load_arrays(fs))
            b.solve(eps_rel=0.0, max_iter=100, check_every=50, precision=opf.PREC_FP32)
            sh = b.shape(opf.PREC_FP32)
            assert sh["ok"] == 1 and sh["k_inst"] == LANE and sh["warps"] == warps and sh["cluster"] > 1
            st = b.status()
            assert np.all(st["iters"] == 100)
            got = [b.locals(j) for j in range(n)]
    for j, g in enumerate(fs):
        ref = oracle_admm.admm(oracle_admm.Prepared(lindist.build(g)), rho=100.0, max_iter=100, check_every=0)
        assert rel_err(got[j][0], ref.xs) <= 1e-4, j
        assert rel_err(got[j][1], ref.lam) <= 1e-4, j


@pytest.mark.parametrize("name,seed,n", [("34", 5034, 5), ("123", 2002, 6)])
def test_lane_converged_objective(name, seed, n):
    f = synth.preset_feeder(name, seed)
    fs = scenarios(f, [4200 + j for j in range(n)])
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n) as b:
            b.set_shape(opf.PREC_FP32, LANE, 16)
            b.set_loads(0, *load_arrays(fs))
            ok = b.solve(precision=opf.PREC_MIXED)
            st = b.status()
            _, obj = b.solution()
    assert ok and np.all(st["converged"]) and np.all(st["pres"] <= 1e-4)
    for j, g in enumerate(fs):
        star, _ = oracle_admm.lp_optimum(lindist.build(g))
        assert abs(obj[j] - star) <= 1e-6 * abs(star), (j, obj[j], star)


def test_lane_instance_alone_equals_in_batch():
    f = synth.preset_feeder("123", 2001)
    n = 130
    fs = scenarios(f, [4900 + j for j in range(n)])
    lp, lq = load_arrays(fs)
    picks = [0, 37, 127, 128, 129]
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, n) as b:
            b.set_shape(opf.PREC_FP32, LANE, 16)
            b.set_shape(opf.PREC_FP64, 4)
            b.set_loads(0, lp, lq)
            assert b.solve(precision=opf.PREC_MIXED, eps_rel=1e-6)
            st = b.status()
            many = {j: (int(st["iters"][j]), *b.locals(j)) for j in picks}
            assert len(set(st["iters"].tolist())) > 1            # stopped at different iterations
        for j in picks:
            with opf.Batch(s, 1) as b1:
                b1.set_shape(opf.PREC_FP32, LANE, 16)
                b1.set_shape(opf.PREC_FP64, 4)
                b1.set_loads(0, lp[j:j + 1], lq[j:j + 1])
                assert b1.solve(precision=opf.PREC_MIXED, eps_rel=1e-6)
                one = (int(b1.status()["iters"][0]), *b1.locals(0))
            assert one[0] == many[j][0], j
            assert np.array_equal(one[1], many[j][1]), j
            assert np.array_equal(one[2], many[j][2]), j


def test_lane_refuses_a_model_too_large():
    f = synth.preset_feeder("8500", 3001)
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        with opf.Batch(s, 1) as b:
            b.set_shape(opf.PREC_FP32, LANE, 16)
            b.set_loads(0, f["load_a"][None], f["load_b"][None])
            with pytest.raises(opf.OPFError) as e:
                b.solve(eps_rel=0.0, max_iter=20, check_every=10, precision=opf.PREC_FP32)
            assert e.value.code == opf.OPF_E_CAPACITY
