"""Thin Python binding of the C ABI in ``include/opf.h`` (argument marshalling only).

Every computation runs inside ``libopf.so``; this module only converts numpy
arrays to pointers.  There is no fallback: if the library is missing or cannot
be loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libopf.so")

OPF_OK = 0
OPF_NOT_CONVERGED = 1
OPF_E_INVALID = -1
OPF_E_INFEASIBLE_LOCAL = -2
OPF_E_STATE = -3
OPF_E_OOM = -4
OPF_E_NUMERIC = -5
OPF_E_TIMEOUT = -6
OPF_E_CUDA = -7
OPF_E_CAPACITY = -8

PREC_FP64, PREC_FP32, PREC_MIXED = 0, 1, 2
ENGINE_AUTO, ENGINE_GRID, ENGINE_CTA, ENGINE_WARP, ENGINE_PERSISTENT = 0, 1, 2, 3, 4
ENGINE_CLUSTER = ENGINE_CTA
SOLVE_HOST_LOOP = 1
SOLVE_TEST_BARRIER_TIMEOUT = 2

_P = C.c_void_p


class Feeder(C.Structure):
    _fields_ = [
        ("n_bus", C.c_int32), ("bus_phases", _P), ("bus_wmin", _P), ("bus_wmax", _P),
        ("bus_gsh", _P), ("bus_bsh", _P),
        ("n_line", C.c_int32), ("line_from", _P), ("line_to", _P), ("line_phases", _P),
        ("line_r", _P), ("line_x", _P), ("line_gs_from", _P), ("line_bs_from", _P),
        ("line_gs_to", _P), ("line_bs_to", _P), ("line_tap", _P),
        ("n_load", C.c_int32), ("load_bus", _P), ("load_phases", _P), ("load_delta", _P),
        ("load_a", _P), ("load_b", _P), ("load_alpha", _P), ("load_beta", _P),
        ("n_gen", C.c_int32), ("gen_bus", _P), ("gen_phases", _P), ("gen_pmin", _P),
        ("gen_pmax", _P), ("gen_qmin", _P), ("gen_qmax", _P), ("gen_cost", _P),
    ]


class Options(C.Structure):
    _fields_ = [("device", C.c_int32), ("stream", _P)]


class SolveOpts(C.Structure):
    _fields_ = [("rho", C.c_double), ("eps_rel", C.c_double), ("eps_abs_pres", C.c_double),
                ("max_iter", C.c_int32), ("check_every", C.c_int32), ("precision", C.c_int32),
                ("recenter_every", C.c_int32), ("engine", C.c_int32), ("flags", C.c_int32),
                ("cluster", C.c_int32)]


class Sizes(C.Structure):
    _fields_ = [("n_global", C.c_int64), ("n_sub", C.c_int64), ("n_slots", C.c_int64),
                ("n_rows", C.c_int64), ("sum_nf", C.c_int64), ("max_ns", C.c_int64),
                ("h2d_bytes", C.c_int64)]


class ServerOpts(C.Structure):
    _fields_ = [("rho", C.c_double), ("eps_rel", C.c_double), ("eps_abs_pres", C.c_double),
                ("max_iter", C.c_int32), ("check_every", C.c_int32), ("chunk_iters", C.c_int32),
                ("keep_solutions", C.c_int32), ("mem_budget", C.c_int64), ("polish_chunk_iters", C.c_int32),
                ("reserved", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libopf.so (built by ``paper_2310_09410_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libopf.so not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    H = C.c_void_p
    lib.opf_create.argtypes = [C.POINTER(Feeder), C.POINTER(Options), C.POINTER(H)]
    lib.opf_create_generic.argtypes = [C.c_int32, _P, _P, _P, _P, C.c_int32, _P, _P, _P, _P, _P,
                                       C.POINTER(Options), C.POINTER(H)]
    lib.opf_precompute.argtypes = [H]
    lib.opf_solve.argtypes = [H, C.c_double, C.c_double, C.c_int32]
    lib.opf_solve_ex.argtypes = [H, C.POINTER(SolveOpts)]
    lib.opf_step.argtypes = [H, C.c_double, C.c_int32]
    lib.opf_reset.argtypes = [H]
    lib.opf_get_solution.argtypes = [H, _P, C.c_size_t, C.POINTER(C.c_double)]
    lib.opf_get_residuals.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    lib.opf_get_locals.argtypes = [H, _P, _P, C.c_size_t]
    lib.opf_set_locals.argtypes = [H, _P, _P, C.c_size_t]
    lib.opf_get_sizes.argtypes = [H, C.POINTER(Sizes)]
    lib.opf_get_timing.argtypes = [H, _P, C.c_int]
    lib.opf_destroy.argtypes = [H]
    lib.opf_destroy.restype = None
    lib.opf_strerror.argtypes = [C.c_int]
    lib.opf_strerror.restype = C.c_char_p
    lib.opf_last_error.argtypes = []
    lib.opf_last_error.restype = C.c_char_p
    lib.opf_global_update_static.argtypes = [C.c_int32, _P, _P, _P, _P, _P, C.c_double, _P, _P, _P]
    lib.opf_batch_create.argtypes = [H, C.c_int32, C.POINTER(H)]
    lib.opf_batch_set_rhs.argtypes = [H, C.c_int32, C.c_int32, _P]
    lib.opf_batch_set_loads.argtypes = [H, C.c_int32, C.c_int32, _P, _P]
    lib.opf_batch_set_loads_device.argtypes = [H, C.c_int32, C.c_int32, _P, _P]
    lib.opf_batch_solve.argtypes = [H, C.POINTER(SolveOpts)]
    lib.opf_batch_step.argtypes = [H, C.c_double, C.c_int32]
    lib.opf_batch_set_shape.argtypes = [H, C.c_int32, C.c_int32, C.c_int32]
    lib.opf_batch_get_shape.argtypes = [H, C.c_int32, _P, C.c_int32]
    lib.opf_batch_get_solution.argtypes = [H, C.c_int32, C.c_int32, _P, _P]
    lib.opf_batch_get_status.argtypes = [H, C.c_int32, C.c_int32, _P, _P, _P]
    lib.opf_batch_get_locals.argtypes = [H, C.c_int32, _P, _P]
    lib.opf_batch_get_timing.argtypes = [H, _P, C.c_int32]
    lib.opf_batch_get_tune_log.argtypes = [H, _P, C.c_int32]
    lib.opf_batch_destroy.argtypes = [H]
    lib.opf_batch_destroy.restype = None
    lib.opf_set_loads.argtypes = [H, _P, _P]
    lib.opf_server_create.argtypes = [C.POINTER(ServerOpts), C.POINTER(H)]
    lib.opf_server_add_model.argtypes = [H, _P, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
    lib.opf_server_submit.argtypes = [H, C.c_int32, _P, _P, C.c_int64]
    lib.opf_server_set_model_tolerance.argtypes = [H, C.c_int32, C.c_double, C.c_double]
    lib.opf_server_set_model_shape.argtypes = [H, C.c_int32, C.c_int32, C.c_int32]
    lib.opf_server_step.argtypes = [H]
    lib.opf_server_poll.argtypes = [H, _P, _P, _P, _P, _P, C.c_int32]
    lib.opf_server_poll_ex.argtypes = [H, _P, _P, _P, _P, _P, _P, C.c_int32]
    lib.opf_batch_set_start.argtypes = [H, _P, _P]
    lib.opf_server_set_model_start.argtypes = [H, C.c_int32, _P, _P]
    lib.opf_server_set_admission.argtypes = [H, C.c_int32, C.c_int32, C.c_double, C.c_double]
    lib.opf_server_model_stats.argtypes = [H, C.c_int32, _P, C.c_int32]
    lib.opf_server_take_solution.argtypes = [H, C.c_int64, _P, C.c_int32]
    lib.opf_server_stats.argtypes = [H, _P, C.c_int32]
    lib.opf_server_destroy.argtypes = [H]
    lib.opf_server_destroy.restype = None
    lib.opf_stream_create_partition.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p),
                                                C.POINTER(C.c_int32)]
    lib.opf_stream_destroy_partition.argtypes = [C.c_void_p]
    lib.opf_probe_fma.argtypes = [C.c_int32, C.c_int32, C.c_int32, _P, _P, C.POINTER(C.c_double)]
    lib.opf_probe_dfma.argtypes = [C.c_int32, C.c_int32, C.c_int32, _P, _P, C.POINTER(C.c_double)]
    lib.opf_batch_set_tmem.argtypes = [H, C.c_int32]
    lib.opf_partition.argtypes = [C.POINTER(Feeder), C.c_int32, _P, C.c_int32]
    lib.opf_shard_create.argtypes = [C.POINTER(Feeder), _P, C.c_int32, C.c_int32, C.POINTER(Options), C.POINTER(H)]
    lib.opf_shard_precompute.argtypes = [H]
    lib.opf_shard_sizes.argtypes = [H, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.opf_shard_maps.argtypes = [H, _P, _P]
    lib.opf_shard_partial.argtypes = [H, C.c_double, _P]
    lib.opf_shard_step.argtypes = [H, C.c_double, _P, _P]
    lib.opf_shard_get_x.argtypes = [H, _P]
    lib.opf_shard_get_locals.argtypes = [H, _P, _P, C.c_size_t]
    lib.opf_shard_stream.argtypes = [H]
    lib.opf_shard_stream.restype = C.c_void_p
    lib.opf_shard_destroy.argtypes = [H]
    lib.opf_shard_destroy.restype = None
    lib.opf_test_rule.argtypes = [_P, C.c_double, C.c_double, C.c_double, _P]
    for name in ("opf_create", "opf_create_generic", "opf_precompute", "opf_solve", "opf_solve_ex",
                 "opf_step", "opf_reset", "opf_get_solution", "opf_get_residuals", "opf_get_locals",
                 "opf_set_locals", "opf_get_sizes", "opf_get_timing", "opf_global_update_static",
                 "opf_batch_create", "opf_batch_set_rhs", "opf_batch_set_loads", "opf_batch_set_loads_device",
                 "opf_batch_solve",
                 "opf_batch_step", "opf_batch_set_shape", "opf_batch_get_shape", "opf_batch_get_solution",
                 "opf_batch_get_status", "opf_batch_get_locals", "opf_batch_get_timing",
                 "opf_batch_get_tune_log", "opf_set_loads", "opf_server_create", "opf_server_add_model",
                 "opf_server_submit", "opf_server_step", "opf_server_poll", "opf_server_take_solution",
                 "opf_server_stats", "opf_stream_create_partition", "opf_stream_destroy_partition",
                 "opf_probe_fma", "opf_server_poll_ex", "opf_server_set_admission", "opf_server_model_stats",
                 "opf_batch_set_start", "opf_server_set_model_start", "opf_batch_set_tmem", "opf_partition",
                 "opf_shard_create", "opf_shard_precompute", "opf_shard_sizes", "opf_shard_maps",
                 "opf_shard_partial", "opf_shard_step", "opf_shard_get_x", "opf_shard_get_locals",
                 "opf_test_rule", "opf_probe_dfma", "opf_server_set_model_tolerance", "opf_server_set_model_shape"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


class OPFError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = lib.opf_strerror(code).decode()
        detail = lib.opf_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}) {detail}")
        self.code = code


def _check(code, where, ok=(OPF_OK,)):
    if code not in ok:
        raise OPFError(code, where)
    return code


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def global_update_static(n, seg_off_ptr, u_ptr, c_ptr, lb_ptr, ub_ptr, rho, x_ptr, obj_ptr, stream=None):
    """Allocation-free global update on caller device pointers (see include/opf.h)."""
    _check(load().opf_global_update_static(int(n), seg_off_ptr, u_ptr, c_ptr, lb_ptr, ub_ptr, float(rho),
                                           x_ptr, obj_ptr, stream), "opf_global_update_static")


def probe_fma(blocks, threads, iters, out_ptr, stream=None):
    """Enqueue the FP32 FMA throughput probe (see include/opf.h); returns its flop count."""
    fl = C.c_double()
    _check(load().opf_probe_fma(int(blocks), int(threads), int(iters), out_ptr, stream, C.byref(fl)),
           "opf_probe_fma")
    return fl.value


def _feeder_struct(f):
    """opf_feeder over numpy copies of the feeder dict's arrays (kept alive
    by the returned dict)."""
    keep = {}

    def arr(name, dtype, shape=None):
        a = np.ascontiguousarray(f[name], dtype=dtype)
        if shape is not None:
            a = a.reshape(shape)
        keep[name] = a
        return _ptr(a)

    nb, nl, nd, ng = int(f["n_bus"]), len(f["line_from"]), len(f["load_bus"]), len(f["gen_bus"])
    fd = Feeder()
    fd.n_bus = nb
    fd.bus_phases = arr("bus_phases", np.uint8)
    fd.bus_wmin = arr("bus_wmin", np.float64, (nb * 3,))
    fd.bus_wmax = arr("bus_wmax", np.float64, (nb * 3,))
    fd.bus_gsh = arr("bus_gsh", np.float64, (nb * 3,))
    fd.bus_bsh = arr("bus_bsh", np.float64, (nb * 3,))
    fd.n_line = nl
    fd.line_from = arr("line_from", np.int32)
    fd.line_to = arr("line_to", np.int32)
    fd.line_phases = arr("line_phases", np.uint8)
    fd.line_r = arr("line_r", np.float64, (nl * 9,))
    fd.line_x = arr("line_x", np.float64, (nl * 9,))
    fd.line_gs_from = arr("line_gs_from", np.float64, (nl * 3,))
    fd.line_bs_from = arr("line_bs_from", np.float64, (nl * 3,))
    fd.line_gs_to = arr("line_gs_to", np.float64, (nl * 3,))
    fd.line_bs_to = arr("line_bs_to", np.float64, (nl * 3,))
    fd.line_tap = arr("line_tap", np.float64, (nl * 3,))
    fd.n_load = nd
    fd.load_bus = arr("load_bus", np.int32)
    fd.load_phases = arr("load_phases", np.uint8)
    fd.load_delta = arr("load_delta", np.uint8)
    fd.load_a = arr("load_a", np.float64, (nd * 3,))
    fd.load_b = arr("load_b", np.float64, (nd * 3,))
    fd.load_alpha = arr("load_alpha", np.float64, (nd * 3,))
    fd.load_beta = arr("load_beta", np.float64, (nd * 3,))
    fd.n_gen = ng
    fd.gen_bus = arr("gen_bus", np.int32)
    fd.gen_phases = arr("gen_phases", np.uint8)
    fd.gen_pmin = arr("gen_pmin", np.float64, (ng * 3,))
    fd.gen_pmax = arr("gen_pmax", np.float64, (ng * 3,))
    fd.gen_qmin = arr("gen_qmin", np.float64, (ng * 3,))
    fd.gen_qmax = arr("gen_qmax", np.float64, (ng * 3,))
    fd.gen_cost = arr("gen_cost", np.float64)
    return fd, keep


def probe_dfma(blocks, threads, iters, out_ptr, stream=None):
    """Enqueue the FP64 FMA throughput probe (see include/opf.h); returns its flop count."""
    fl = C.c_double()
    _check(load().opf_probe_dfma(int(blocks), int(threads), int(iters), out_ptr, stream, C.byref(fl)),
           "opf_probe_dfma")
    return fl.value


class Solver:
    """One problem instance on one device (wraps an ``opf_handle``)."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    # ---------------------------------------------------------- creation
    @classmethod
    def from_feeder(cls, f, device=0, stream=None):
        lib = load()
        fd, keep = _feeder_struct(f)
        opts = Options(int(device), C.c_void_p(stream) if stream else None)
        h = C.c_void_p()
        _check(lib.opf_create(C.byref(fd), C.byref(opts), C.byref(h)), "opf_create")
        return cls(h, keep)

    @classmethod
    def from_generic(cls, c, lb, ub, subs, is_voltage=None, device=0, stream=None):
        """subs: list of dicts with "idx", "A" (m x n) and "b"."""
        lib = load()
        c = np.ascontiguousarray(c, np.float64)
        lb = np.ascontiguousarray(lb, np.float64)
        ub = np.ascontiguousarray(ub, np.float64)
        volt = None if is_voltage is None else np.ascontiguousarray(is_voltage, np.uint8)
        m_s = np.array([np.asarray(s["A"]).reshape(-1, len(s["idx"])).shape[0] for s in subs], np.int32)
        n_s = np.array([len(s["idx"]) for s in subs], np.int32)
        A = np.ascontiguousarray(np.concatenate([np.asarray(s["A"], np.float64).ravel() for s in subs]
                                                + [np.zeros(0)]))
        b = np.ascontiguousarray(np.concatenate([np.asarray(s["b"], np.float64).ravel() for s in subs]
                                                + [np.zeros(0)]))
        idx = np.ascontiguousarray(np.concatenate([np.asarray(s["idx"], np.int64) for s in subs]).astype(np.int32))
        keep = dict(c=c, lb=lb, ub=ub, volt=volt, m_s=m_s, n_s=n_s, A=A, b=b, idx=idx)
        opts = Options(int(device), C.c_void_p(stream) if stream else None)
        h = C.c_void_p()
        _check(lib.opf_create_generic(len(c), _ptr(c), _ptr(lb), _ptr(ub), _ptr(volt), len(subs),
                                      _ptr(m_s), _ptr(n_s), _ptr(A), _ptr(b), _ptr(idx),
                                      C.byref(opts), C.byref(h)), "opf_create_generic")
        return cls(h, keep)

    # ---------------------------------------------------------- calls
    def precompute(self):
        _check(load().opf_precompute(self._h), "opf_precompute")

    def solve(self, rho=100.0, eps_rel=1e-8, eps_abs_pres=1e-4, max_iter=1_000_000, check_every=50,
              precision=PREC_FP64, recenter_every=0, engine=ENGINE_AUTO, flags=0, cluster=0):
        o = SolveOpts(rho, eps_rel, eps_abs_pres, int(max_iter), int(check_every), int(precision),
                      int(recenter_every), int(engine), int(flags), int(cluster))
        rc = load().opf_solve_ex(self._h, C.byref(o))
        _check(rc, "opf_solve_ex", ok=(OPF_OK, OPF_NOT_CONVERGED))
        return rc == OPF_OK

    def solve_simple(self, rho=100.0, eps=1e-8, max_iter=1_000_000):
        rc = load().opf_solve(self._h, rho, eps, int(max_iter))
        _check(rc, "opf_solve", ok=(OPF_OK, OPF_NOT_CONVERGED))
        return rc == OPF_OK

    def step(self, n_iters, rho=100.0):
        _check(load().opf_step(self._h, rho, int(n_iters)), "opf_step")

    def reset(self):
        _check(load().opf_reset(self._h), "opf_reset")

    def sizes(self):
        s = Sizes()
        _check(load().opf_get_sizes(self._h, C.byref(s)), "opf_get_sizes")
        return {k: int(getattr(s, k)) for k, _ in Sizes._fields_}

    def solution(self):
        n = self.sizes()["n_global"]
        x = np.zeros(n)
        obj = C.c_double()
        _check(load().opf_get_solution(self._h, _ptr(x), n, C.byref(obj)), "opf_get_solution")
        return x, obj.value

    def residuals(self):
        p, d, ep, ed = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        it = C.c_int64()
        _check(load().opf_get_residuals(self._h, C.byref(p), C.byref(d), C.byref(ep), C.byref(ed),
                                        C.byref(it)), "opf_get_residuals")
        return {"pres": p.value, "dres": d.value, "eps_prim": ep.value, "eps_dual": ed.value,
                "iters": it.value}

    def locals(self):
        L = self.sizes()["n_slots"]
        xs, lam = np.zeros(L), np.zeros(L)
        _check(load().opf_get_locals(self._h, _ptr(xs), _ptr(lam), L), "opf_get_locals")
        return xs, lam

    def set_locals(self, xs, lam):
        xs = np.ascontiguousarray(xs, np.float64)
        lam = np.ascontiguousarray(lam, np.float64)
        _check(load().opf_set_locals(self._h, _ptr(xs), _ptr(lam), len(xs)), "opf_set_locals")

    def set_loads(self, load_p, load_q):
        """New load values ([n_load, 3] each); precompute() again before iterating."""
        lp = np.ascontiguousarray(load_p, np.float64)
        lq = np.ascontiguousarray(load_q, np.float64)
        _check(load().opf_set_loads(self._h, _ptr(lp), _ptr(lq)), "opf_set_loads")

    def timing(self):
        t = np.zeros(6)
        _check(load().opf_get_timing(self._h, _ptr(t), 6), "opf_get_timing")
        return {"precompute_ms": t[0], "iterate_ms": t[1], "polish_ms": t[2],
                "main_iters": int(t[3]), "polish_iters": int(t[4]), "recenters": int(t[5])}

    def close(self):
        if self._h:
            load().opf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many instances of one model (wraps an ``opf_batch``): every instance
    shares the solver's A_s, c and bounds and has its own right-hand side."""

    def __init__(self, solver: "Solver", n_inst: int):
        lib = load()
        h = C.c_void_p()
        _check(lib.opf_batch_create(solver._h, int(n_inst), C.byref(h)), "opf_batch_create")
        self._b = h
        self._solver = solver           # the batch refers to the handle: keep it alive
        self.n = int(n_inst)
        sz = solver.sizes()
        self.n_global, self.n_slots, self.n_rows = sz["n_global"], sz["n_slots"], sz["n_rows"]

    def set_rhs(self, first, rhs):
        rhs = np.ascontiguousarray(rhs, np.float64).reshape(-1, self.n_rows)
        _check(load().opf_batch_set_rhs(self._b, int(first), rhs.shape[0], _ptr(rhs)), "opf_batch_set_rhs")

    def set_loads(self, first, load_p, load_q):
        """load_p, load_q: [count, n_load, 3] (like feeder load_a / load_b)."""
        lp = np.ascontiguousarray(load_p, np.float64)
        lq = np.ascontiguousarray(load_q, np.float64)
        if lp.shape != lq.shape or lp.ndim != 3 or lp.shape[2] != 3:
            raise ValueError("load arrays must both be [count, n_load, 3]")
        _check(load().opf_batch_set_loads(self._b, int(first), lp.shape[0], _ptr(lp), _ptr(lq)),
               "opf_batch_set_loads")

    def set_loads_device(self, first, count, load_p_ptr, load_q_ptr):
        """Device pointers to [count, n_load, 3] doubles each (e.g. torch tensors' data_ptr())."""
        _check(load().opf_batch_set_loads_device(self._b, int(first), int(count), load_p_ptr, load_q_ptr),
               "opf_batch_set_loads_device")

    def set_shape(self, precision, k_inst=0, warps=0):
        _check(load().opf_batch_set_shape(self._b, int(precision), int(k_inst), int(warps)), "opf_batch_set_shape")

    def shape(self, precision=PREC_FP32):
        out = np.zeros(11, np.int32)
        _check(load().opf_batch_get_shape(self._b, int(precision), _ptr(out), 11), "opf_batch_get_shape")
        keys = ("ok", "k_inst", "warps", "chunks_per_lane", "tasks", "chunks", "smem_bytes", "ctas", "tmem",
                "tmem_cols", "cluster")
        return {k: int(v) for k, v in zip(keys, out)}

    def set_tmem(self, enable):
        """FP32 engine: lambda and bbar~ in tensor memory (True) or streamed from L2."""
        _check(load().opf_batch_set_tmem(self._b, int(bool(enable))), "opf_batch_set_tmem")

    def solve(self, rho=100.0, eps_rel=1e-8, eps_abs_pres=1e-4, max_iter=1_000_000, check_every=50,
              precision=PREC_MIXED, recenter_every=0, flags=0):
        o = SolveOpts(rho, eps_rel, eps_abs_pres, int(max_iter), int(check_every), int(precision),
                      int(recenter_every), 0, int(flags), 0)
        rc = load().opf_batch_solve(self._b, C.byref(o))
        _check(rc, "opf_batch_solve", ok=(OPF_OK, OPF_NOT_CONVERGED))
        return rc == OPF_OK

    def step(self, n_iters, rho=100.0):
        _check(load().opf_batch_step(self._b, float(rho), int(n_iters)), "opf_batch_step")

    def solution(self, first=0, count=None, out=None):
        """x [count, n_global] and objectives [count]; out = (x, obj) writes into
        caller arrays (e.g. views of pinned host memory) instead of new ones."""
        count = self.n - first if count is None else count
        if out is None:
            x = np.zeros((count, self.n_global))
            obj = np.zeros(count)
        else:
            x, obj = out
            if (x.shape != (count, self.n_global) or obj.shape != (count,) or x.dtype != np.float64
                    or obj.dtype != np.float64 or not x.flags.c_contiguous or not obj.flags.c_contiguous):
                raise ValueError("out must be C-contiguous float64 arrays [count, n_global] and [count]")
        _check(load().opf_batch_get_solution(self._b, int(first), int(count), _ptr(x), _ptr(obj)),
               "opf_batch_get_solution")
        return x, obj

    def status(self, first=0, count=None):
        count = self.n - first if count is None else count
        res = np.zeros((count, 4))
        it = np.zeros(count, np.int32)
        conv = np.zeros(count, np.int32)
        _check(load().opf_batch_get_status(self._b, int(first), int(count), _ptr(res), _ptr(it), _ptr(conv)),
               "opf_batch_get_status")
        return {"pres": res[:, 0], "dres": res[:, 1], "eps_prim": res[:, 2], "eps_dual": res[:, 3],
                "iters": it, "converged": conv.astype(bool)}

    def set_start(self, xs=None, lam=None):
        """Warm start of instances set afterwards (None: the Sec. V-A point)."""
        if xs is None:
            _check(load().opf_batch_set_start(self._b, None, None), "opf_batch_set_start")
            return
        xs = np.ascontiguousarray(xs, np.float64)
        lam = np.ascontiguousarray(lam, np.float64)
        _check(load().opf_batch_set_start(self._b, _ptr(xs), _ptr(lam)), "opf_batch_set_start")

    def locals(self, inst):
        xs, lam = np.zeros(self.n_slots), np.zeros(self.n_slots)
        _check(load().opf_batch_get_locals(self._b, int(inst), _ptr(xs), _ptr(lam)), "opf_batch_get_locals")
        return xs, lam

    def timing(self):
        t = np.zeros(8)
        _check(load().opf_batch_get_timing(self._b, _ptr(t), 8), "opf_batch_get_timing")
        return {"fp32_ms": t[0], "fp64_ms": t[1], "tune_ms": t[2], "mean_iters": t[3], "converged": int(t[4]),
                "fp32_passes": int(t[5]), "fp64_passes": int(t[6]), "engine_ms": t[7]}

    def tune_log(self):
        lib = load()
        n = lib.opf_batch_get_tune_log(self._b, None, 0)
        out = np.zeros(max(n, 1))
        lib.opf_batch_get_tune_log(self._b, _ptr(out), n)
        return [(int(out[i]), int(out[i + 1]), float(out[i + 2])) for i in range(0, n, 3)]

    def close(self):
        if self._b:
            load().opf_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching request server (wraps an ``opf_server``)."""

    def __init__(self, rho=100.0, eps_rel=1e-8, eps_abs_pres=1e-4, max_iter=1_000_000, check_every=50,
                 chunk_iters=1000, keep_solutions=False, mem_budget=0, polish_chunk_iters=0):
        lib = load()
        o = ServerOpts(rho, eps_rel, eps_abs_pres, int(max_iter), int(check_every), int(chunk_iters),
                       int(bool(keep_solutions)), int(mem_budget), int(polish_chunk_iters), 0)
        h = C.c_void_p()
        _check(lib.opf_server_create(C.byref(o), C.byref(h)), "opf_server_create")
        self._s = h
        self._solvers = []             # the server refers to the handles: keep them alive
        self._n_global = {}

    def add_model(self, solvers, capacity):
        """solvers: precomputed Solver objects of one feeder topology."""
        solvers = list(solvers)
        arr = (C.c_void_p * len(solvers))(*[sv._h.value if isinstance(sv._h, C.c_void_p) else sv._h
                                            for sv in solvers])
        mid = C.c_int32()
        _check(load().opf_server_add_model(self._s, C.cast(arr, C.c_void_p), len(solvers), int(capacity),
                                           C.byref(mid)), "opf_server_add_model")
        self._solvers.extend(solvers)
        self._n_global[mid.value] = solvers[0].sizes()["n_global"]
        return mid.value

    def set_model_shape(self, model, k_inst=0, warps=0):
        _check(load().opf_server_set_model_shape(self._s, int(model), int(k_inst), int(warps)),
               "opf_server_set_model_shape")

    def set_model_tolerance(self, model, eps_rel, eps_abs_pres=1e-4):
        _check(load().opf_server_set_model_tolerance(self._s, int(model), float(eps_rel), float(eps_abs_pres)),
               "opf_server_set_model_tolerance")

    def set_model_start(self, model, xs=None, lam=None):
        if xs is None:
            _check(load().opf_server_set_model_start(self._s, int(model), None, None), "opf_server_set_model_start")
            return
        xs = np.ascontiguousarray(xs, np.float64)
        lam = np.ascontiguousarray(lam, np.float64)
        _check(load().opf_server_set_model_start(self._s, int(model), _ptr(xs), _ptr(lam)),
               "opf_server_set_model_start")

    def set_admission(self, model, max_queue=0, max_wait_s=0.0, max_service_s=0.0):
        _check(load().opf_server_set_admission(self._s, int(model), int(max_queue), float(max_wait_s),
                                               float(max_service_s)), "opf_server_set_admission")

    def submit(self, model, load_p, load_q, tag, refusable=False):
        """Queue a request; with refusable=True a refusal by the model's
        admission policy returns False instead of raising."""
        lp = np.ascontiguousarray(load_p, np.float64)
        lq = np.ascontiguousarray(load_q, np.float64)
        rc = load().opf_server_submit(self._s, int(model), _ptr(lp), _ptr(lq), int(tag))
        if refusable and rc == OPF_E_CAPACITY:
            return False
        _check(rc, "opf_server_submit")
        return True

    def step(self):
        _check(load().opf_server_step(self._s), "opf_server_step")

    def poll(self, max_n=4096):
        tags = np.zeros(max_n, np.int64)
        conv = np.zeros(max_n, np.int32)
        obj = np.zeros(max_n)
        it = np.zeros(max_n, np.int32)
        lat = np.zeros(max_n)
        sts = np.zeros(max_n, np.int32)
        n = load().opf_server_poll_ex(self._s, _ptr(tags), _ptr(sts), _ptr(conv), _ptr(obj), _ptr(it), _ptr(lat),
                                      int(max_n))
        if n < 0:
            raise OPFError(n, "opf_server_poll_ex")
        return [{"tag": int(tags[i]), "status": int(sts[i]), "converged": bool(conv[i]),
                 "objective": float(obj[i]), "iters": int(it[i]), "latency_s": float(lat[i])} for i in range(n)]

    def take_solution(self, tag, model):
        x = np.zeros(self._n_global[model])
        _check(load().opf_server_take_solution(self._s, int(tag), _ptr(x), len(x)), "opf_server_take_solution")
        return x

    def stats(self):
        out = np.zeros(7, np.int64)
        _check(load().opf_server_stats(self._s, _ptr(out), 7), "opf_server_stats")
        keys = ("submitted", "polled", "queued", "running", "slots", "passes", "mem_bytes")
        return {k: int(v) for k, v in zip(keys, out)}

    def model_stats(self, model):
        out = np.zeros(10, np.int64)
        _check(load().opf_server_model_stats(self._s, int(model), _ptr(out), 10), "opf_server_model_stats")
        keys = ("submitted", "served", "converged", "refused", "shed", "queued", "running", "slots")
        d = {k: int(v) for k, v in zip(keys, out)}
        d["service_s"] = float(out[8]) / 1e6
        d["stopped"] = int(out[9])
        return d

    def close(self):
        if self._s:
            load().opf_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class SMPartition:
    """A stream confined to a subset of the device's SMs (green context).
    n_sm > 0: that many SMs; n_sm < 0: all but -n_sm SMs."""

    def __init__(self, n_sm, device=0, priority=0):
        st = C.c_void_p()
        cnt = C.c_int32()
        _check(load().opf_stream_create_partition(int(device), int(n_sm), int(priority), C.byref(st), C.byref(cnt)),
               "opf_stream_create_partition")
        self.stream = st.value
        self.sm_count = cnt.value

    def close(self):
        if self.stream:
            load().opf_stream_destroy_partition(C.c_void_p(self.stream))
            self.stream = None


def partition(f, n_parts, n_sub):
    """Part of each of the feeder model's n_sub subsystems (opf_partition)."""
    fd, keep = _feeder_struct(f)
    out = np.zeros(n_sub, np.int32)
    _check(load().opf_partition(C.byref(fd), int(n_parts), _ptr(out), int(n_sub)), "opf_partition")
    return out


def apply_test_rule(sums, rho, eps_rel, eps_abs_pres):
    """Sec. III-C test on summed squares (opf_test_rule): (converged, [pres,
    dres, eps_prim / eps_rel, eps_dual / eps_rel, objective])."""
    sm = np.ascontiguousarray(sums, np.float64)
    out = np.zeros(5)
    rc = load().opf_test_rule(_ptr(sm), float(rho), float(eps_rel), float(eps_abs_pres), _ptr(out))
    if rc < 0:
        raise OPFError(rc, "opf_test_rule")
    return bool(rc), out


class Shard:
    """One part of a sharded instance (wraps an ``opf_shard``); the caller
    exchanges the cut sums between partial() and step()."""

    def __init__(self, f, sub_part, part, device=0, stream=None):
        fd, self._keep = _feeder_struct(f)
        sp = np.ascontiguousarray(sub_part, np.int32)
        self._keep["sub_part"] = sp
        opts = Options(int(device), C.c_void_p(stream) if stream else None)
        h = C.c_void_p()
        _check(load().opf_shard_create(C.byref(fd), _ptr(sp), len(sp), int(part), C.byref(opts), C.byref(h)),
               "opf_shard_create")
        self._s = h
        g, c, l = C.c_int32(), C.c_int32(), C.c_int32()
        _check(load().opf_shard_sizes(h, C.byref(g), C.byref(c), C.byref(l)), "opf_shard_sizes")
        self.n_global, self.n_cut, self.n_slots = g.value, c.value, l.value
        self.global_of_local = np.zeros(self.n_global, np.int32)
        self.cut_global = np.zeros(max(self.n_cut, 1), np.int32)
        _check(load().opf_shard_maps(h, _ptr(self.global_of_local), _ptr(self.cut_global)), "opf_shard_maps")
        self.cut_global = self.cut_global[:self.n_cut]
        self.stream = load().opf_shard_stream(h)

    def precompute(self):
        _check(load().opf_shard_precompute(self._s), "opf_shard_precompute")

    def partial(self, rho, sig_ptr):
        _check(load().opf_shard_partial(self._s, float(rho), sig_ptr), "opf_shard_partial")

    def step(self, rho, sig_tot_ptr, sums_ptr=None):
        _check(load().opf_shard_step(self._s, float(rho), sig_tot_ptr, sums_ptr), "opf_shard_step")

    def x(self):
        out = np.zeros(self.n_global)
        _check(load().opf_shard_get_x(self._s, _ptr(out)), "opf_shard_get_x")
        return out

    def locals(self):
        xs, lam = np.zeros(self.n_slots), np.zeros(self.n_slots)
        _check(load().opf_shard_get_locals(self._s, _ptr(xs), _ptr(lam), self.n_slots), "opf_shard_get_locals")
        return xs, lam

    def close(self):
        if self._s:
            load().opf_shard_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
