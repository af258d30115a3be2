"""opf_global_update_static: the allocation-free global update.

Some callers cannot allocate device memory: control loops that forbid
allocation once they run (an allocation may block, or fail when memory is
short, at any moment), and hosts whose device memory is handed out only by
their own allocator.  For them the library offers the global update and the
objective c^T x on caller device arrays, with its scratch in a fixed device
array instead of memory from a handle.  Its results must equal what
opf_get_solution returns for the same iterate, on two calls in a row (the
shared scratch keeps the previous call's contents), and a call after the
first in a context must leave the device's free memory unchanged.

This file is named to be collected last.
"""
import numpy as np
import pytest

from oracle import lindist
from paper_2310_09410_gb300 import opf, synth

pytestmark = pytest.mark.gpu

TOL = 1e-10   # relative, as the FP64 parity tests


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def reference_and_inputs(name, seed, steps, rho=100.0):
    """x and c^T x from opf_get_solution after `steps` iterations, and the
    grouped u = rho x_s - lambda of the iterate that produced them."""
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    gidx = np.concatenate([s["idx"] for s in M.subs])          # canonical slot -> global
    with opf.Solver.from_feeder(f) as s:
        s.precompute()
        s.step(steps - 1, rho=rho)
        xs, lam = s.locals()
        s.step(1, rho=rho)
        x_ref, obj_ref = s.solution()
    order = np.argsort(gidx, kind="stable")
    u = (rho * xs - lam)[order]
    seg = np.concatenate([[0], np.cumsum(np.bincount(gidx, minlength=M.n))]).astype(np.int32)
    return M, seg, u, x_ref, obj_ref


def call_static(torch, M, seg, u, rho=100.0, stream=None, free_out=None):
    dev = torch.device("cuda", 0)
    t = {
        "seg": torch.from_numpy(seg).to(dev),
        "u": torch.from_numpy(np.ascontiguousarray(u)).to(dev),
        "c": torch.from_numpy(np.ascontiguousarray(M.c)).to(dev),
        "lb": torch.from_numpy(np.ascontiguousarray(M.lb)).to(dev),
        "ub": torch.from_numpy(np.ascontiguousarray(M.ub)).to(dev),
        "x": torch.full((M.n,), float("nan"), dtype=torch.float64, device=dev),
        "obj": torch.full((1,), float("nan"), dtype=torch.float64, device=dev),
    }
    torch.cuda.synchronize()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    if free_out is not None:
        free_out.append(torch.cuda.mem_get_info(0)[0])
    opf.global_update_static(M.n, t["seg"].data_ptr(), t["u"].data_ptr(), t["c"].data_ptr(),
                             t["lb"].data_ptr(), t["ub"].data_ptr(), rho, t["x"].data_ptr(),
                             t["obj"].data_ptr(), stream)
    torch.cuda.synchronize()
    if free_out is not None:
        free_out.append(torch.cuda.mem_get_info(0)[0])
    return t["x"].cpu().numpy(), float(t["obj"].cpu().numpy()[0])


def test_matches_get_solution_on_two_calls():
    torch = pytest.importorskip("torch")
    cases = [("123", 2001, 37), ("13", 1001, 120)]   # larger first: the second call reuses less scratch
    free = []
    for k, (name, seed, steps) in enumerate(cases):
        M, seg, u, x_ref, obj_ref = reference_and_inputs(name, seed, steps)
        x, obj = call_static(torch, M, seg, u, free_out=free if k == 1 else None)
        assert np.all(np.isfinite(x))
        assert np.max(np.abs(x - x_ref)) <= TOL * max(1.0, float(np.max(np.abs(x_ref))))
        assert abs(obj - obj_ref) <= TOL * max(1.0, abs(obj_ref))
    assert free[0] == free[1], "the second call changed the device's free memory"


def test_matches_get_solution_on_sm_partition_stream():
    """A stream of an SM partition runs its kernels in its own context; the
    call looks the scratch up in that context and gives the same results."""
    torch = pytest.importorskip("torch")
    M, seg, u, x_ref, obj_ref = reference_and_inputs("123", 2001, 21)
    part = opf.SMPartition(32)
    try:
        for _ in range(2):
            x, obj = call_static(torch, M, seg, u, stream=part.stream)
            assert np.max(np.abs(x - x_ref)) <= TOL * max(1.0, float(np.max(np.abs(x_ref))))
            assert abs(obj - obj_ref) <= TOL * max(1.0, abs(obj_ref))
    finally:
        part.close()


def test_rejects_bad_arguments_without_launching():
    opf.load()
    with pytest.raises(opf.OPFError) as e:
        opf.global_update_static(opf_max_globals() + 1, 1, 1, 1, 1, 1, 100.0, 1, 1)
    assert e.value.code == opf.OPF_E_CAPACITY
    with pytest.raises(opf.OPFError) as e:
        opf.global_update_static(10, None, 1, 1, 1, 1, 100.0, 1, 1)
    assert e.value.code == opf.OPF_E_INVALID
    with pytest.raises(opf.OPFError) as e:
        opf.global_update_static(10, 1, 1, 1, 1, 1, -1.0, 1, 1)
    assert e.value.code == opf.OPF_E_INVALID


def opf_max_globals():
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "opf.h")).read()
    blocks = int(re.search(r"#define OPF_STATIC_MAX_BLOCKS (\d+)", text).group(1))
    return 256 * blocks
