"""C ABI: the library builds, loads, exports every declared entry point, and
rejects malformed input on the host before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2310_09410_gb300 import build, opf, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return opf.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(opf_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    raw = ctypes.CDLL(opf.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_strerror_names_every_code(lib):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.opf_strerror(code).decode() != "unknown status"
    assert lib.opf_strerror(42).decode() == "unknown status"


def _bad(f, **changes):
    g = dict(f)
    g.update(changes)
    return g


@pytest.mark.parametrize("mutate", [
    lambda f: _bad(f, line_to=np.array([2] + list(f["line_to"][1:]), dtype=np.int32)),  # bus with two feeders
    lambda f: _bad(f, line_from=np.array([1] + list(f["line_from"][1:]), dtype=np.int32)),   # self loop
    lambda f: _bad(f, bus_phases=np.array([7] + [1] * (f["n_bus"] - 1), dtype=np.uint8)),
    lambda f: _bad(f, load_bus=np.array([f["n_bus"] + 3] + list(f["load_bus"][1:]), dtype=np.int32)),
    lambda f: _bad(f, gen_pmin=np.full_like(f["gen_pmin"], 1.0), gen_pmax=np.zeros_like(f["gen_pmax"])),
    lambda f: _bad(f, load_delta=np.ones(len(f["load_bus"]), dtype=np.uint8)),   # delta on 1-phase bus
])
def test_malformed_feeder_rejected_on_host(lib, mutate):
    f = synth.preset_feeder("13", 1001)
    with pytest.raises(opf.OPFError) as e:
        opf.Solver.from_feeder(mutate(f))
    assert e.value.code == opf.OPF_E_INVALID


def test_generic_validation_on_host(lib):
    g = synth.random_generic(1)
    subs = [dict(s) for s in g["subs"]]
    subs[0] = dict(subs[0], idx=np.array([0, 0] + list(subs[0]["idx"][2:]), dtype=np.int32))
    with pytest.raises(opf.OPFError) as e:
        opf.Solver.from_generic(g["c"], g["lb"], g["ub"], subs)
    assert e.value.code == opf.OPF_E_INVALID
    big = [{"idx": np.arange(300), "A": np.ones((1, 300)), "b": np.ones(1)}]
    with pytest.raises(opf.OPFError) as e:
        opf.Solver.from_generic(np.zeros(300), -np.ones(300), np.ones(300), big)
    assert e.value.code == opf.OPF_E_CAPACITY
    uncovered = [{"idx": np.arange(5), "A": np.ones((1, 5)), "b": np.ones(1)}]
    with pytest.raises(opf.OPFError) as e:
        opf.Solver.from_generic(np.zeros(6), -np.ones(6), np.ones(6), uncovered)
    assert e.value.code == opf.OPF_E_INVALID


def test_batch_entry_points_reject_bad_handles_on_host(lib):
    out = ctypes.c_void_p()
    lib.opf_batch_create.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.opf_batch_create(None, 4, ctypes.byref(out)) == opf.OPF_E_INVALID
    assert lib.opf_batch_solve(None, None) == opf.OPF_E_INVALID
    assert lib.opf_batch_step(None, 100.0, 10) == opf.OPF_E_INVALID
    assert lib.opf_batch_set_shape(None, opf.PREC_FP32, 8, 16) == opf.OPF_E_INVALID
    assert lib.opf_batch_get_status(None, 0, 1, None, None, None) == opf.OPF_E_INVALID
    assert lib.opf_batch_set_loads(None, 0, 1, None, None) == opf.OPF_E_INVALID
    lib.opf_batch_destroy(None)                      # a no-op


def test_server_options_and_handles_checked_on_host(lib):
    o = opf.ServerOpts(100.0, 1e-8, 1e-4, 1000, 50, 1000, 0, 0)
    out = ctypes.c_void_p()
    bad = [opf.ServerOpts(-1.0, 1e-8, 1e-4, 1000, 50, 1000, 0, 0),      # rho
           opf.ServerOpts(100.0, 1e-8, 1e-4, 1000, 3, 1000, 0, 0),       # odd check interval
           opf.ServerOpts(100.0, 1e-8, 1e-4, 1000, 50, 1010, 0, 0),      # chunk not a multiple
           opf.ServerOpts(100.0, 1e-8, 1e-4, 1000, 50, 1000, 0, -5),     # budget
           opf.ServerOpts(100.0, 1e-8, 1e-4, 1000, 50, 1000, 0, 0, 75)]  # polish interval not a multiple
    for b in bad:
        assert lib.opf_server_create(ctypes.byref(b), ctypes.byref(out)) == opf.OPF_E_INVALID
    assert lib.opf_server_create(ctypes.byref(o), ctypes.byref(out)) == opf.OPF_OK
    z = np.zeros(3)
    assert lib.opf_server_submit(out, 0, z.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p),
                                 7) == opf.OPF_E_INVALID                 # no model 0
    st = np.zeros(7, np.int64)
    assert lib.opf_server_stats(out, st.ctypes.data_as(ctypes.c_void_p), 7) == opf.OPF_OK
    assert list(st[:5]) == [0, 0, 0, 0, 0]
    assert lib.opf_server_poll(out, None, None, None, None, None, 16) == 0
    assert lib.opf_server_step(out) == opf.OPF_OK                        # nothing to do
    lib.opf_server_set_model_tolerance.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_double]
    assert lib.opf_server_set_model_tolerance(out, 0, 1e-9, 1e-4) == opf.OPF_E_INVALID   # no model 0
    lib.opf_server_destroy(out)


def test_fma_probe_rejects_bad_sizes_on_host(lib):
    from paper_2310_09410_gb300 import opf
    for blocks, threads, iters in ((0, 256, 1), (1, 48, 1), (1, 2048, 1), (1, 256, 0)):
        with pytest.raises(opf.OPFError) as e:
            opf.probe_fma(blocks, threads, iters, 1)
        assert e.value.code == opf.OPF_E_INVALID


@pytest.mark.gpu
def test_fma_probe_measures_a_plausible_fp32_rate():
    """The roofline's denominator: the probe's flop count is the one its
    kernel performs (8 chains x 16 x iters FMAs per thread, 2 flops each) and
    its timed rate lies between a tenth of and the nominal FP32 peak."""
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_09410_gb300 import opf
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(2 * sms * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        opf.probe_fma(2 * sms, 1024, 512, out.data_ptr(), stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fl = opf.probe_fma(2 * sms, 1024, 512, out.data_ptr(), stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    assert fl == 2.0 * 8 * 16 * 512 * 1024 * 2 * sms
    tflops = fl / (e0.elapsed_time(e1) / 1e3) / 1e12
    nominal = sms * 128 * 2 * 2.1e9 / 1e12
    assert 0.1 * nominal < tflops < 1.05 * nominal, (tflops, nominal)
    assert torch.isfinite(out).all()


@pytest.mark.gpu
def test_fp64_fma_probe_counts_its_flops():
    """The FP64 probe (the denominator of FP64 iterations): its flop count and
    a rate of the order of this part's FP64 FMA throughput."""
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_09410_gb300 import opf
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(sms * 1024, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    opf.probe_dfma(sms, 1024, 8, out.data_ptr(), stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fl = opf.probe_dfma(sms, 1024, 8, out.data_ptr(), stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    assert fl == 2.0 * 8 * 16 * 8 * 1024 * sms
    tflops = fl / (e0.elapsed_time(e1) / 1e3) / 1e12
    assert 0.05 < tflops < 10.0, tflops
    assert torch.isfinite(out).all()
