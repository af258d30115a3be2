"""ORACLE (test infrastructure only): FP64 ADMM of Algorithm 1 and the LP it solves.

Only tests, the smoke check and the CPU-baseline leg of the benchmark may
import this module.  Pieces, each following the passage it cites:

* ``precompute``   -- Abar_s and bbar_s of Eq. closed_2, written literally as
  A^T (A A^T)^{-1} A - I and A^T (A A^T)^{-1} b (Sec. III-B); a rank-deficient
  A_s is first row-reduced (the preprocessing step the paper names), keeping a
  maximal independent row set chosen by pivoted QR and checking that the
  dropped rows are consistent;
* ``init_point``   -- the starting point of Sec. V-A: lambda = 0, a local copy
  is 1 for a squared-voltage variable, the midpoint of its bounds when both are
  finite, 0 when it has none (one finite bound: that bound, a reading the
  paper leaves open);
* ``admm``         -- Algorithm 1 itself, run by the plain C loop in
  ``admm_ref.c`` (global update Eq. closed_1, local update Eq. closed_2, dual
  update Eq. ADMM-3, residuals and stopping test of Sec. III-C);
* ``lp_optimum``   -- the centralized LP of Eq. LP_model solved directly by a
  library LP solver (HiGHS through scipy), the value ADMM must converge to;
* ``dense_ipm``    -- a hand-written dense primal-dual interior-point solver
  for the same bounded LP, for tiny instances.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import lindist

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "admm_ref.c")
_LIB = os.path.join(_HERE, "_admm_ref.so")
_lib = None


def build_lib(force=False):
    """Compile the C loop (gcc, -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        P = ctypes.c_void_p
        lib.oracle_admm.restype = ctypes.c_int
        lib.oracle_admm.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int, P, P, P, P, P,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, P, P, P, P, P]
        _lib = lib
    return _lib


def precompute(A, b, tol=1e-12):
    """(Abar, bbar) of Eq. closed_2 for one subsystem (Sec. III-B)."""
    import scipy.linalg as sla
    A = np.asarray(A, dtype=float)
    b = np.asarray(b, dtype=float)
    n = A.shape[1]
    if A.shape[0] == 0:
        return -np.eye(n), np.zeros(n)
    # row reduction: a maximal independent set of rows (pivoted QR of A^T)
    _, R, piv = sla.qr(A.T, pivoting=True, mode="economic")
    diag = np.abs(np.diag(R)) if R.size else np.zeros(0)
    scale = max(np.linalg.norm(A), 1.0)
    rank = int(np.sum(diag > tol * scale))
    keep = np.sort(piv[:rank])
    Ar, br = A[keep], b[keep]
    G = Ar @ Ar.T
    Abar = Ar.T @ np.linalg.solve(G, Ar) - np.eye(n)
    bbar = Ar.T @ np.linalg.solve(G, br)
    if rank < A.shape[0]:
        if np.linalg.norm(A @ bbar - b) > 1e-9 * max(np.linalg.norm(b), 1.0):
            raise ValueError("inconsistent local system A_s x_s = b_s")
    return Abar, bbar


def init_point(M):
    """Value every local copy of global i starts from (Sec. V-A)."""
    lb, ub = M.lb, M.ub
    x0 = np.zeros(M.n)
    for i in range(M.n):
        if M.is_voltage[i]:
            x0[i] = 1.0
        elif np.isfinite(lb[i]) and np.isfinite(ub[i]):
            x0[i] = 0.5 * (lb[i] + ub[i])
        elif np.isfinite(lb[i]):
            x0[i] = lb[i]
        elif np.isfinite(ub[i]):
            x0[i] = ub[i]
    return x0


class Prepared:
    """Subsystems flattened for the C loop: slot offsets, global index of each
    slot, dense Abar_s blocks and bbar."""

    def __init__(self, M):
        self.M = M
        ns = [len(s["idx"]) for s in M.subs]
        self.off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
        self.gidx = np.concatenate([s["idx"] for s in M.subs]).astype(np.int32)
        blocks, bb = [], []
        for s in M.subs:
            Ab, bbar = precompute(s["A"], s["b"])
            blocks.append(Ab.ravel())
            bb.append(bbar)
        self.abar = np.concatenate(blocks)
        self.aoff = np.concatenate([[0], np.cumsum([n * n for n in ns])]).astype(np.int64)
        self.bbar = np.concatenate(bb)
        self.x0 = init_point(M)


class Result:
    pass


def admm(M_or_prep, rho=100.0, eps_rel=1e-8, eps_abs_pres=1e-4, max_iter=10000,
         check_every=1, record=False, xs=None, lam=None):
    """Run Algorithm 1 from the Sec. V-A start (or from given xs, lam).

    With ``check_every = 0`` exactly ``max_iter`` iterations run.  Stopping
    test (Sec. III-C with an absolute gate): pres <= eps_rel * max(|Bx|, |x_s|),
    dres <= eps_rel * |lambda| and pres <= eps_abs_pres.
    """
    P = M_or_prep if isinstance(M_or_prep, Prepared) else Prepared(M_or_prep)
    M = P.M
    L = int(P.off[-1])
    xs = (P.x0[P.gidx].copy() if xs is None else np.array(xs, dtype=float, copy=True))
    lam = (np.zeros(L) if lam is None else np.array(lam, dtype=float, copy=True))
    x = np.zeros(M.n)
    hist = np.zeros((max(max_iter, 1), 5)) if record else None
    conv = ctypes.c_int(0)
    lib = _load()
    c = np.ascontiguousarray(M.c, dtype=float)
    lb = np.ascontiguousarray(M.lb, dtype=float)
    ub = np.ascontiguousarray(M.ub, dtype=float)

    def p(a):
        return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None

    it = lib.oracle_admm(M.n, p(c), p(lb), p(ub), len(M.subs), p(P.off), p(P.gidx),
                         p(P.abar), p(P.aoff), p(P.bbar), rho, eps_rel, eps_abs_pres,
                         int(max_iter), int(check_every), p(xs), p(lam), p(x), p(hist),
                         ctypes.byref(conv))
    if it < 0:
        raise ValueError("a global variable has no local copy")
    r = Result()
    r.x, r.xs, r.lam, r.iters, r.converged = x, xs, lam, it, bool(conv.value)
    r.objective = float(M.c @ x)
    r.hist = hist[:it] if record else None
    if it > 0:
        if record:
            r.pres, r.dres = float(hist[it - 1, 0]), float(hist[it - 1, 1])
        else:
            xg = x[P.gidx]
            r.pres = float(np.linalg.norm(xg - xs))
            r.dres = float("nan")
    return r


def lp_optimum(M):
    """Optimal value and point of the centralized LP (Eq. LP_model) by HiGHS."""
    import scipy.sparse as sp
    from scipy.optimize import linprog
    A, b = lindist.centralized(M)
    res = linprog(M.c, A_eq=sp.csr_matrix(A), b_eq=b, bounds=list(zip(M.lb, M.ub)),
                  method="highs", options={"primal_feasibility_tolerance": 1e-10,
                                           "dual_feasibility_tolerance": 1e-10})
    if res.status != 0:
        raise ValueError("centralized LP not solved: " + str(res.message))
    return float(res.fun), res.x


def dense_ipm(c, A, b, lb, ub, tol=1e-12, max_iter=200):
    """Hand-written dense primal-dual interior-point method (Mehrotra
    predictor-corrector) for  min c^T x  s.t.  A x = b,  lb <= x <= ub.

    KKT conditions with slacks for the finite bounds:
        A x = b,  x - s_l = lb,  x + s_u = ub,  c - A^T y - z_l + z_u = 0,
        s_l z_l = mu,  s_u z_u = mu,  (s, z) >= 0,
    Newton steps on the augmented system [[D, -A^T], [A, 0]] with
    D = z_l / s_l + z_u / s_u (free variables have D = 0).  Rows of A are
    assumed independent.  Returns (objective, x).
    """
    c = np.asarray(c, float)
    A = np.asarray(A, float)
    b = np.asarray(b, float)
    n, m = len(c), A.shape[0]
    hl, hu = np.isfinite(lb), np.isfinite(ub)
    L = np.where(hl, lb, 0.0)
    U = np.where(hu, ub, 0.0)
    x = np.where(hl & hu, 0.5 * (L + U), np.where(hl, L + 1.0, np.where(hu, U - 1.0, 0.0)))
    one_l, one_u = np.where(hl, 1.0, 0.0), np.where(hu, 1.0, 0.0)
    sl = np.where(hl, np.maximum(x - L, 1e-2), 1.0)
    su = np.where(hu, np.maximum(U - x, 1e-2), 1.0)
    zl, zu = one_l.copy(), one_u.copy()
    y = np.zeros(m)
    nb = max(int(hl.sum() + hu.sum()), 1)
    for _ in range(max_iter):
        rp = b - A @ x
        rl = (L + sl - x) * one_l
        ru = (U - su - x) * one_u
        rd = c - A.T @ y - zl + zu
        mu = float((sl * zl * one_l).sum() + (su * zu * one_u).sum()) / nb
        if (np.linalg.norm(rp) <= tol * (1 + np.linalg.norm(b)) and
                np.linalg.norm(rd) <= tol * (1 + np.linalg.norm(c)) and
                np.linalg.norm(rl) + np.linalg.norm(ru) <= tol and mu <= tol):
            break
        D = (zl / sl) * one_l + (zu / su) * one_u
        K = np.zeros((n + m, n + m))
        K[:n, :n] = np.diag(D + 1e-13)
        K[:n, n:] = -A.T
        K[n:, :n] = A
        K[n:, n:] = -1e-13 * np.eye(m)

        def newton(target_l, target_u):
            # s_l dz_l + z_l ds_l = target_l - s_l z_l (same for u); ds_l = dx - rl, ds_u = ru - dx
            cl = (target_l - sl * zl) * one_l
            cu = (target_u - su * zu) * one_u
            h = -rd + (cl + zl * rl) / sl * one_l + (zu * ru - cu) / su * one_u
            sol = np.linalg.solve(K, np.concatenate([h, rp]))
            dx, dy = sol[:n], sol[n:]
            dsl = (dx - rl) * one_l
            dsu = (ru - dx) * one_u
            dzl = (cl - zl * dsl) / sl * one_l
            dzu = (cu - zu * dsu) / su * one_u
            return dx, dy, dsl, dsu, dzl, dzu

        def max_step(v, dv, mask):
            mm = mask & (dv < 0)
            return min(1.0, float(np.min(-v[mm] / dv[mm]))) if np.any(mm) else 1.0

        dx, dy, dsl, dsu, dzl, dzu = newton(0.0, 0.0)
        ap = min(max_step(sl, dsl, hl), max_step(su, dsu, hu))
        ad = min(max_step(zl, dzl, hl), max_step(zu, dzu, hu))
        mu_aff = float(((sl + ap * dsl) * (zl + ad * dzl) * one_l).sum() +
                       ((su + ap * dsu) * (zu + ad * dzu) * one_u).sum()) / nb
        sigma = (mu_aff / mu) ** 3 if mu > 0 else 0.0
        dx, dy, dsl, dsu, dzl, dzu = newton(sigma * mu - dsl * dzl, sigma * mu - dsu * dzu)
        ap = min(1.0, 0.995 * min(max_step(sl, dsl, hl), max_step(su, dsu, hu)))
        ad = min(1.0, 0.995 * min(max_step(zl, dzl, hl), max_step(zu, dzu, hu)))
        x, sl, su = x + ap * dx, sl + ap * dsl, su + ap * dsu
        y, zl, zu = y + ad * dy, zl + ad * dzl, zu + ad * dzu
    return float(c @ x), x
