"""ORACLE (test infrastructure only): LinDist3Flow LP and its decomposition.

Only tests, the smoke check and the CPU-baseline leg of the benchmark may
import this module.  It is a plain, slow, obviously-correct restatement of

* the linearized unbalanced OPF of Sec. II-A (operational bounds, power
  balance, voltage-dependent load model VDLM-1..10, linearized line flow with
  the 3x3 matrices M^p and M^q), written as the abstract LP
  ``min c^T x  s.t.  A x = b,  lb <= x <= ub``  (Eq. LP_model);
* the componentwise decomposition of Sec. V-A: one subsystem per bus and per
  line, a leaf bus merged into the line that feeds it, giving the consensus
  form of Eq. OurModel: local systems ``A_s x_s = b_s`` with ``x_s = B_s x``.

Canonical orderings (an interface shared with the CUDA library, which has its
own implementation of the same rules):

* global variables, in the order of the x listing under Eq. LP_model:
  generators (per gen, per phase: p^g, q^g), buses (per bus, per phase: w),
  loads (per load, per phase: p^b, q^b, p^d, q^d), lines (per line, per phase:
  p_eij, q_eij, p_eji, q_eji); phases ascending a, b, c;
* subsystems: every non-leaf bus in bus order, then every line in line order
  (a line whose to-bus is a leaf carries that bus's rows too);
* local variables of a subsystem: ascending global index.

The rows inside a subsystem are in no particular order; the projection the
method uses depends only on the affine set they describe.
"""
from __future__ import annotations

import math

import numpy as np

SQ3 = math.sqrt(3.0)
INF = math.inf


def phases(mask):
    return [p for p in range(3) if (int(mask) >> p) & 1]


def mp_mq(r, x):
    """M^p and M^q of a line (Sec. II-A, Eq. power_flow_eqns), from the 3x3
    resistance r and reactance x, exactly as the two printed matrices."""
    mp = np.array([
        [-2 * r[0, 0], r[0, 1] - SQ3 * x[0, 1], r[0, 2] + SQ3 * x[0, 2]],
        [r[1, 0] + SQ3 * x[1, 0], -2 * r[1, 1], r[1, 2] - SQ3 * x[1, 2]],
        [r[2, 0] - SQ3 * x[2, 0], r[2, 1] + SQ3 * x[2, 1], -2 * r[2, 2]],
    ])
    mq = np.array([
        [-2 * x[0, 0], x[0, 1] + SQ3 * r[0, 1], x[0, 2] - SQ3 * r[0, 2]],
        [x[1, 0] - SQ3 * r[1, 0], -2 * x[1, 1], x[1, 2] + SQ3 * r[1, 2]],
        [x[2, 0] + SQ3 * r[2, 0], x[2, 1] - SQ3 * r[2, 1], -2 * x[2, 2]],
    ])
    return mp, mq


class Model:
    """The LP of Eq. LP_model plus the subsystems of Eq. OurModel."""

    def __init__(self):
        self.names = []        # (kind, owner, phase, field) per global variable
        self.lb = []
        self.ub = []
        self.c = []
        self.is_voltage = []
        self.subs = []         # dicts: kind, idx (sorted global ids), A, b


def _index_variables(f, M):
    gen_v, bus_v, load_v, line_v = {}, {}, {}, {}

    def add(name, lo, hi, cost=0.0, volt=False):
        M.names.append(name)
        M.lb.append(lo)
        M.ub.append(hi)
        M.c.append(cost)
        M.is_voltage.append(volt)
        return len(M.names) - 1

    for k in range(len(f["gen_bus"])):
        for p in phases(f["gen_phases"][k]):
            gen_v[k, p, "p"] = add(("gen", k, p, "p"), f["gen_pmin"][k, p], f["gen_pmax"][k, p], f["gen_cost"][k])
            gen_v[k, p, "q"] = add(("gen", k, p, "q"), f["gen_qmin"][k, p], f["gen_qmax"][k, p])
    for i in range(f["n_bus"]):
        for p in phases(f["bus_phases"][i]):
            bus_v[i, p] = add(("bus", i, p, "w"), f["bus_wmin"][i, p], f["bus_wmax"][i, p], volt=True)
    for l in range(len(f["load_bus"])):
        for p in phases(f["load_phases"][l]):
            for fld in ("pb", "qb", "pd", "qd"):
                load_v[l, p, fld] = add(("load", l, p, fld), -INF, INF)
    for e in range(len(f["line_from"])):
        for p in phases(f["line_phases"][e]):
            for fld in ("pij", "qij", "pji", "qji"):
                line_v[e, p, fld] = add(("line", e, p, fld), -INF, INF)
    return gen_v, bus_v, load_v, line_v


def _adjacency(f):
    nb = f["n_bus"]
    adj = {"out": [[] for _ in range(nb)], "in": [[] for _ in range(nb)],
           "load": [[] for _ in range(nb)], "gen": [[] for _ in range(nb)]}
    for e in range(len(f["line_from"])):
        adj["out"][int(f["line_from"][e])].append(e)
        adj["in"][int(f["line_to"][e])].append(e)
    for l in range(len(f["load_bus"])):
        adj["load"][int(f["load_bus"][l])].append(l)
    for k in range(len(f["gen_bus"])):
        adj["gen"][int(f["gen_bus"][k])].append(k)
    return adj


def _bus_rows(f, adj, i, bus_v, gen_v, load_v, line_v):
    """Rows owned by bus i: power balance (Eq. balance_eqns) and the rows of
    its loads (VDLM-1..10).  Each row is (dict var->coef, rhs)."""
    rows = []
    for p in phases(f["bus_phases"][i]):
        rp, rq = {}, {}
        for e in adj["out"][i]:
            if p in phases(f["line_phases"][e]):
                rp[line_v[e, p, "pij"]] = 1.0
                rq[line_v[e, p, "qij"]] = 1.0
        for e in adj["in"][i]:
            if p in phases(f["line_phases"][e]):
                rp[line_v[e, p, "pji"]] = 1.0
                rq[line_v[e, p, "qji"]] = 1.0
        for l in adj["load"][i]:
            if p in phases(f["load_phases"][l]):
                rp[load_v[l, p, "pb"]] = 1.0
                rq[load_v[l, p, "qb"]] = 1.0
        rp[bus_v[i, p]] = rp.get(bus_v[i, p], 0.0) + f["bus_gsh"][i, p]
        rq[bus_v[i, p]] = rq.get(bus_v[i, p], 0.0) - f["bus_bsh"][i, p]
        for k in adj["gen"][i]:
            if p in phases(f["gen_phases"][k]):
                rp[gen_v[k, p, "p"]] = -1.0
                rq[gen_v[k, p, "q"]] = -1.0
        rows.append((rp, 0.0))
        rows.append((rq, 0.0))
    for l in adj["load"][i]:
        delta = bool(f["load_delta"][l])
        ph = phases(f["load_phases"][l])
        wfac = 3.0 if delta else 1.0   # VDLM-3 / VDLM-4
        for p in ph:
            a, b = f["load_a"][l, p], f["load_b"][l, p]
            al, be = f["load_alpha"][l, p], f["load_beta"][l, p]
            # VDLM-1: p^d = (a alpha / 2)(w_hat - 1) + a
            rows.append(({load_v[l, p, "pd"]: 1.0, bus_v[i, p]: -0.5 * a * al * wfac}, a - 0.5 * a * al))
            # VDLM-2: q^d = (b beta / 2)(w_hat - 1) + b
            rows.append(({load_v[l, p, "qd"]: 1.0, bus_v[i, p]: -0.5 * b * be * wfac}, b - 0.5 * b * be))
        if not delta:
            for p in ph:   # VDLM-5
                rows.append(({load_v[l, p, "pb"]: 1.0, load_v[l, p, "pd"]: -1.0}, 0.0))
                rows.append(({load_v[l, p, "qb"]: 1.0, load_v[l, p, "qd"]: -1.0}, 0.0))
        else:
            if ph != [0, 1, 2]:
                raise ValueError("a delta load needs all three phases")
            pb = [load_v[l, p, "pb"] for p in range(3)]
            qb = [load_v[l, p, "qb"] for p in range(3)]
            pd = [load_v[l, p, "pd"] for p in range(3)]
            qd = [load_v[l, p, "qd"] for p in range(3)]
            # VDLM-6
            r = {}
            for p in range(3):
                r[pb[p]] = 1.0
                r[pd[p]] = -1.0
            rows.append((r, 0.0))
            r = {}
            for p in range(3):
                r[qb[p]] = 1.0
                r[qd[p]] = -1.0
            rows.append((r, 0.0))
            # VDLM-7..10 (phase 1, 2, 3 of the paper = index 0, 1, 2), all moved to the left side
            rows.append(({pb[1]: 1.5, qb[1]: -SQ3 / 2, pd[1]: -1.0, pd[0]: -0.5, qd[0]: SQ3 / 2}, 0.0))
            rows.append(({pb[1]: SQ3 / 2, qb[1]: 1.5, pd[0]: -SQ3 / 2, qd[0]: -0.5, qd[1]: -1.0}, 0.0))
            rows.append(({qb[1]: SQ3, pb[2]: 1.5, qb[2]: -SQ3 / 2, pd[0]: -0.5, qd[0]: -SQ3 / 2, pd[2]: -1.0}, 0.0))
            rows.append(({pb[1]: -SQ3, pb[2]: SQ3 / 2, qb[2]: 1.5, pd[0]: SQ3 / 2, qd[0]: -0.5, qd[2]: -1.0}, 0.0))
    return rows


def _line_rows(f, e, bus_v, line_v):
    """Rows owned by line e = (i, j): Eq. power_flow_eqns for every phase."""
    i, j = int(f["line_from"][e]), int(f["line_to"][e])
    ph = phases(f["line_phases"][e])
    mp, mq = mp_mq(f["line_r"][e], f["line_x"][e])
    gi, gj = f["line_gs_from"][e], f["line_gs_to"][e]
    bi, bj = f["line_bs_from"][e], f["line_bs_to"][e]
    tau = f["line_tap"][e]
    rows = []
    for p in ph:
        # p_eij + p_eji = g_ij w_i + g_ji w_j
        rows.append(({line_v[e, p, "pij"]: 1.0, line_v[e, p, "pji"]: 1.0,
                      bus_v[i, p]: -gi[p], bus_v[j, p]: -gj[p]}, 0.0))
        # q_eij + q_eji = -b_ij w_i - b_ji w_j
        rows.append(({line_v[e, p, "qij"]: 1.0, line_v[e, p, "qji"]: 1.0,
                      bus_v[i, p]: bi[p], bus_v[j, p]: bj[p]}, 0.0))
        # w_i = tau w_j - sum_psi Mp (p_ij - g_ij w_i) - sum_psi Mq (q_ij + b_ij w_i)
        r = {bus_v[i, p]: 1.0, bus_v[j, p]: -tau[p]}
        for q in ph:
            r[line_v[e, q, "pij"]] = r.get(line_v[e, q, "pij"], 0.0) + mp[p, q]
            r[bus_v[i, q]] = r.get(bus_v[i, q], 0.0) - mp[p, q] * gi[q]
            r[line_v[e, q, "qij"]] = r.get(line_v[e, q, "qij"], 0.0) + mq[p, q]
            r[bus_v[i, q]] = r.get(bus_v[i, q], 0.0) + mq[p, q] * bi[q]
        rows.append((r, 0.0))
    return rows


def _dense(rows, idx):
    pos = {g: k for k, g in enumerate(idx)}
    A = np.zeros((len(rows), len(idx)))
    b = np.zeros(len(rows))
    for r, (coef, rhs) in enumerate(rows):
        for g, v in coef.items():
            A[r, pos[g]] += v
        b[r] = rhs
    return A, b


def check_feeder(f):
    """Radial-feeder checks: one incoming line per non-root bus, none into the
    root, phases nested (line within its from-bus, bus equal to its line)."""
    nb = f["n_bus"]
    to = list(f["line_to"])
    if len(to) != nb - 1 or sorted(to) != list(range(1, nb)):
        raise ValueError("every non-root bus needs exactly one incoming line")
    for e in range(len(to)):
        i, j = int(f["line_from"][e]), int(f["line_to"][e])
        if int(f["line_phases"][e]) & ~int(f["bus_phases"][i]):
            raise ValueError("line phases must be a subset of its from-bus phases")
        if int(f["bus_phases"][j]) != int(f["line_phases"][e]):
            raise ValueError("a bus takes the phases of its incoming line")
    # acyclic: walking up from any bus reaches the root
    par = {int(f["line_to"][e]): int(f["line_from"][e]) for e in range(len(to))}
    for j in range(1, nb):
        seen, k = 0, j
        while k != 0:
            k = par[k]
            seen += 1
            if seen > nb:
                raise ValueError("the lines do not form a tree rooted at bus 0")


def build(f):
    """Feeder dict -> Model (global c, lb, ub and the subsystems)."""
    check_feeder(f)
    M = Model()
    gen_v, bus_v, load_v, line_v = _index_variables(f, M)
    nb = f["n_bus"]
    has_child = np.zeros(nb, dtype=bool)
    for e in range(len(f["line_from"])):
        has_child[int(f["line_from"][e])] = True
    leaf = [i != 0 and not has_child[i] for i in range(nb)]

    adj = _adjacency(f)

    def bus_vars(i):
        s = set()
        for p in phases(f["bus_phases"][i]):
            s.add(bus_v[i, p])
        for e in adj["out"][i]:
            for p in phases(f["line_phases"][e]):
                s |= {line_v[e, p, "pij"], line_v[e, p, "qij"]}
        for e in adj["in"][i]:
            for p in phases(f["line_phases"][e]):
                s |= {line_v[e, p, "pji"], line_v[e, p, "qji"]}
        for l in adj["load"][i]:
            for p in phases(f["load_phases"][l]):
                s |= {load_v[l, p, fld] for fld in ("pb", "qb", "pd", "qd")}
        for k in adj["gen"][i]:
            for p in phases(f["gen_phases"][k]):
                s |= {gen_v[k, p, "p"], gen_v[k, p, "q"]}
        return s

    def line_vars(e):
        s = set()
        i, j = int(f["line_from"][e]), int(f["line_to"][e])
        for p in phases(f["line_phases"][e]):
            s |= {line_v[e, p, fld] for fld in ("pij", "qij", "pji", "qji")}
            s |= {bus_v[i, p], bus_v[j, p]}
        return s

    for i in range(nb):
        if leaf[i]:
            continue
        idx = sorted(bus_vars(i))
        rows = _bus_rows(f, adj, i, bus_v, gen_v, load_v, line_v)
        A, b = _dense(rows, idx)
        M.subs.append({"kind": "bus", "owner": i, "idx": np.array(idx, dtype=np.int64), "A": A, "b": b})
    for e in range(len(f["line_from"])):
        j = int(f["line_to"][e])
        vars_ = line_vars(e)
        rows = _line_rows(f, e, bus_v, line_v)
        kind = "line"
        if leaf[j]:
            vars_ |= bus_vars(j)
            rows += _bus_rows(f, adj, j, bus_v, gen_v, load_v, line_v)
            kind = "leaf"
        idx = sorted(vars_)
        A, b = _dense(rows, idx)
        M.subs.append({"kind": kind, "owner": e, "idx": np.array(idx, dtype=np.int64), "A": A, "b": b})
    M.lb = np.array(M.lb, dtype=float)
    M.ub = np.array(M.ub, dtype=float)
    M.c = np.array(M.c, dtype=float)
    M.is_voltage = np.array(M.is_voltage, dtype=bool)
    M.n = len(M.names)
    M.leaves = int(sum(leaf))
    return M


def centralized(M):
    """Stack every subsystem's rows over the global variables: Eq. LP_model's
    (A, b).  Each equation belongs to exactly one subsystem."""
    rows = sum(s["A"].shape[0] for s in M.subs)
    A = np.zeros((rows, M.n))
    b = np.zeros(rows)
    r = 0
    for s in M.subs:
        m = s["A"].shape[0]
        A[r:r + m, s["idx"]] = s["A"]
        b[r:r + m] = s["b"]
        r += m
    return A, b


def from_generic(g):
    """Model from the random generic consensus instance (synth.random_generic)."""
    M = Model()
    M.n = len(g["c"])
    M.c = np.asarray(g["c"], dtype=float)
    M.lb = np.asarray(g["lb"], dtype=float)
    M.ub = np.asarray(g["ub"], dtype=float)
    M.is_voltage = np.zeros(M.n, dtype=bool)
    M.names = [("generic", i, 0, "x") for i in range(M.n)]
    for s in g["subs"]:
        M.subs.append({"kind": "generic", "owner": 0, "idx": np.asarray(s["idx"], dtype=np.int64),
                       "A": np.asarray(s["A"], dtype=float), "b": np.asarray(s["b"], dtype=float)})
    M.leaves = 0
    return M
