"""Seeded synthetic feeders and load scenarios (input recipe only).

This module builds the *inputs* of the linearized multi-phase OPF: a radial
three-phase distribution feeder with its lines, loads and generators, in the
units the model of Sec. II-A uses (per-unit powers on a 1 MVA-per-phase base,
squared voltage magnitudes in p.u.).  It holds none of the method's
arithmetic: no power-flow equation, no decomposition, no ADMM step.  Both the
CUDA library and the CPU oracle consume its output; neither is imported here.

Recipe (the stand-in for the IEEE 13/37/123/8500 test feeders of Sec. V-A,
which are not available):

* tree by uniform random attachment: node k picks its parent uniformly among
  the earlier nodes whose depth is below ``depth_max``; bus 0 is the
  substation; line ``k-1`` joins ``parent(k)`` (from side) to ``k`` (to side);
* phase set of each line drawn from {abc, ab, bc, a, b, c}, a subset of the
  parent bus's phases; lines leaving the substation are abc; a bus takes the
  phases of the line feeding it; with ``p_single`` given, lines below a
  multi-phase bus go single-phase when a per-line uniform draw is below a
  threshold, bisected so that a fraction ``p_single`` of all lines ends up
  single-phase (otherwise the set is uniform over the allowed ones);
* 3x3 R and X (ohm/km): diagonals U[0.1, 0.6], off-diagonals 0.3-0.5 x the
  mean of the two diagonals, symmetric; length U[0.1, 1] km;
* spot loads on distinct random non-root buses, one per bus phase,
  P U[0, 200] kW per phase, power factor U[0.85, 0.98], constant-power wye
  (alpha = beta = 0);
* one substation source at bus 0 (w fixed to 1, p and q unbounded) and DERs
  on distinct random non-root buses with a box [0, 150] kW and +-100 kvar in
  total, split equally over the bus phases;
* linear cost U[10, 50] per MWh on every generator's active power;
* squared-voltage bounds [0.9025, 1.1025] at every non-root bus;
* an impedance scale ``kappa`` (ohm -> p.u.) chosen so that a conservative
  bound on the squared-voltage deviation with all DERs at zero stays within
  ``vdrop_target``; the bound is sum over the path of
  2 * sum_psi (|r| + |x|) * (P + Q) of the downstream load, which keeps the
  synthetic LP feasible (the per-unit base is not fixed by the paper).
"""
from __future__ import annotations

import math

import numpy as np

PHASE_A, PHASE_B, PHASE_C = 1, 2, 4
ALLOWED_SETS = (7, 3, 6, 1, 2, 4)  # abc, ab, bc, a, b, c
SINGLE_SETS = (1, 2, 4)

W_MIN, W_MAX = 0.9025, 1.1025

# Feeder sizes: name -> (buses, loads, DERs, depth cap, single-phase prob.)
PRESETS = {
    "13": (13, 9, 2, 6, None),
    "34": (34, 24, 4, 12, None),
    "123": (123, 85, 10, 30, 0.4),
    "8500": (8500, 1200, 100, 60, 0.7),
}


def phase_list(mask: int) -> list[int]:
    """Phase indices (0, 1, 2) contained in a bit mask, ascending."""
    return [p for p in range(3) if (int(mask) >> p) & 1]


def _draw_tree(rng, n_bus, depth_max):
    parent = np.full(n_bus, -1, dtype=np.int64)
    depth = np.zeros(n_bus, dtype=np.int64)
    eligible = [0]
    for k in range(1, n_bus):
        p = eligible[rng.integers(len(eligible))]
        parent[k] = p
        depth[k] = depth[p] + 1
        if depth[k] < depth_max:
            eligible.append(k)
    return parent, depth


def make_feeder(n_bus, n_load, n_der, depth_max=6, p_single=None, seed=0,
                vdrop_target=0.068):
    """Draw one radial feeder; returns a dict of numpy arrays (see module doc)."""
    if n_bus < 2:
        raise ValueError("a feeder needs at least two buses")
    rng = np.random.default_rng(seed)
    parent, depth = _draw_tree(rng, n_bus, depth_max)
    n_line = n_bus - 1

    u_single = rng.random(n_bus)   # single-phase draw per line (line k-1 feeds bus k)
    u_pick = rng.random(n_bus)     # which set among the allowed ones

    def assign(q):
        ph = np.zeros(n_bus, dtype=np.uint8)
        ph[0] = 7
        for k in range(1, n_bus):
            pm = int(ph[parent[k]])
            if parent[k] == 0:
                ph[k] = 7
                continue
            allowed = [s for s in ALLOWED_SETS if s & ~pm == 0]
            if q is not None:
                singles = [s for s in allowed if s in SINGLE_SETS]
                multi = [s for s in allowed if s not in SINGLE_SETS]
                allowed = multi if (multi and u_single[k] >= q) else singles
            ph[k] = allowed[int(u_pick[k] * len(allowed))]
        return ph

    if p_single is None:
        bus_ph = assign(None)
    else:
        # realised fraction of single-phase lines grows with the threshold q
        # (a single-phase line forces its subtree single-phase): bisect q so
        # that the fraction of single-phase lines is close to p_single
        lo, hi = 0.0, 1.0
        for _ in range(30):
            mid = 0.5 * (lo + hi)
            frac = float(np.mean([m in SINGLE_SETS for m in assign(mid)[1:]]))
            lo, hi = (mid, hi) if frac < p_single else (lo, mid)
        bus_ph = assign(lo)
    line_from = parent[1:].astype(np.int32)
    line_to = np.arange(1, n_bus, dtype=np.int32)
    line_ph = bus_ph[1:].copy()

    r_ohm = np.zeros((n_line, 3, 3))
    x_ohm = np.zeros((n_line, 3, 3))
    for e in range(n_line):
        length = rng.uniform(0.1, 1.0)
        for mat in (r_ohm, x_ohm):
            d = rng.uniform(0.1, 0.6, size=3)
            z = np.diag(d)
            for a in range(3):
                for b in range(a + 1, 3):
                    z[a, b] = z[b, a] = rng.uniform(0.3, 0.5) * 0.5 * (d[a] + d[b])
            mask = np.array([(int(line_ph[e]) >> p) & 1 for p in range(3)], dtype=float)
            mat[e] = z * length * np.outer(mask, mask)

    n_load = min(n_load, n_bus - 1)
    load_bus = np.sort(rng.choice(np.arange(1, n_bus), size=n_load, replace=False)).astype(np.int32)
    load_ph = bus_ph[load_bus].copy()
    load_a = np.zeros((n_load, 3))
    load_b = np.zeros((n_load, 3))
    for l in range(n_load):
        for p in phase_list(load_ph[l]):
            pkw = rng.uniform(0.0, 200.0)
            pf = rng.uniform(0.85, 0.98)
            load_a[l, p] = pkw / 1000.0
            load_b[l, p] = pkw / 1000.0 * math.tan(math.acos(pf))

    n_der = min(n_der, n_bus - 1)
    der_bus = np.sort(rng.choice(np.arange(1, n_bus), size=n_der, replace=False)).astype(np.int32)
    n_gen = 1 + n_der
    gen_bus = np.concatenate([[0], der_bus]).astype(np.int32)
    gen_ph = np.concatenate([[7], bus_ph[der_bus]]).astype(np.uint8)
    gen_pmin = np.zeros((n_gen, 3))
    gen_pmax = np.zeros((n_gen, 3))
    gen_qmin = np.zeros((n_gen, 3))
    gen_qmax = np.zeros((n_gen, 3))
    gen_pmin[0, :] = -np.inf
    gen_pmax[0, :] = np.inf
    gen_qmin[0, :] = -np.inf
    gen_qmax[0, :] = np.inf
    for g in range(1, n_gen):
        ph = phase_list(gen_ph[g])
        for p in ph:
            gen_pmax[g, p] = 0.150 / len(ph)
            gen_qmin[g, p] = -0.100 / len(ph)
            gen_qmax[g, p] = 0.100 / len(ph)
    gen_cost = rng.uniform(10.0, 50.0, size=n_gen)

    # impedance scale: conservative bound on |w - 1| with the DERs at zero
    down = np.zeros((n_bus, 3))
    for l in range(n_load):
        down[load_bus[l]] += load_a[l] + load_b[l]
    for k in range(n_bus - 1, 0, -1):
        down[parent[k]] += down[k]
    bound = np.zeros(n_bus)
    for k in range(1, n_bus):
        e = k - 1
        z = np.abs(r_ohm[e]) + np.abs(x_ohm[e])
        bound[k] = bound[parent[k]] + 2.0 * float(np.max(z @ down[k]))
    worst = float(bound.max())
    kappa = vdrop_target / worst if worst > 0 else 1.0

    bus_wmin = np.full((n_bus, 3), W_MIN)
    bus_wmax = np.full((n_bus, 3), W_MAX)
    bus_wmin[0, :] = 1.0
    bus_wmax[0, :] = 1.0

    return {
        "n_bus": n_bus,
        "bus_phases": bus_ph,
        "bus_wmin": bus_wmin,
        "bus_wmax": bus_wmax,
        "bus_gsh": np.zeros((n_bus, 3)),
        "bus_bsh": np.zeros((n_bus, 3)),
        "line_from": line_from,
        "line_to": line_to,
        "line_phases": line_ph,
        "line_r": r_ohm * kappa,
        "line_x": x_ohm * kappa,
        "line_gs_from": np.zeros((n_line, 3)),
        "line_bs_from": np.zeros((n_line, 3)),
        "line_gs_to": np.zeros((n_line, 3)),
        "line_bs_to": np.zeros((n_line, 3)),
        "line_tap": np.ones((n_line, 3)),
        "load_bus": load_bus,
        "load_phases": load_ph,
        "load_delta": np.zeros(n_load, dtype=np.uint8),
        "load_a": load_a,
        "load_b": load_b,
        "load_alpha": np.zeros((n_load, 3)),
        "load_beta": np.zeros((n_load, 3)),
        "gen_bus": gen_bus,
        "gen_phases": gen_ph,
        "gen_pmin": gen_pmin,
        "gen_pmax": gen_pmax,
        "gen_qmin": gen_qmin,
        "gen_qmax": gen_qmax,
        "gen_cost": gen_cost,
        "meta": {
            "seed": seed,
            "kappa": kappa,
            "depth": int(depth.max()),
            "leaves": int(sum(1 for k in range(1, n_bus) if not np.any(parent == k))),
        },
    }


def preset_feeder(name: str, seed: int, **kw):
    """One of the named feeder sizes ("13", "34", "123", "8500")."""
    n_bus, n_load, n_der, dmax, p1 = PRESETS[name]
    return make_feeder(n_bus, n_load, n_der, depth_max=dmax, p_single=p1, seed=seed, **kw)


def load_scenario(feeder, seed: int, lo=0.6, hi=1.2, sigma=0.05):
    """Copy of ``feeder`` with its loads scaled by U[lo, hi] x N(1, sigma) per load."""
    rng = np.random.default_rng(seed)
    f = dict(feeder)
    scale = rng.uniform(lo, hi)
    noise = rng.normal(1.0, sigma, size=len(feeder["load_bus"]))
    fac = (scale * noise)[:, None]
    f["load_a"] = feeder["load_a"] * fac
    f["load_b"] = feeder["load_b"] * fac
    f["meta"] = dict(feeder["meta"], scenario_seed=seed, scenario_scale=float(scale))
    return f


def with_zip_delta(feeder, seed: int, p_delta=0.5):
    """Copy of ``feeder`` whose loads get ZIP exponents alpha, beta in {0, 1, 2}
    and, on three-phase buses, a delta connection with probability ``p_delta``."""
    rng = np.random.default_rng(seed)
    f = dict(feeder)
    n = len(feeder["load_bus"])
    f["load_alpha"] = rng.integers(0, 3, size=(n, 3)).astype(float)
    f["load_beta"] = rng.integers(0, 3, size=(n, 3)).astype(float)
    delta = np.zeros(n, dtype=np.uint8)
    for l in range(n):
        if int(feeder["load_phases"][l]) == 7 and rng.random() < p_delta:
            delta[l] = 1
    f["load_delta"] = delta
    return f


def with_shunts_and_taps(feeder, seed: int, g_max=2e-3, b_max=4e-3, tap_dev=0.03):
    """Copy of ``feeder`` with shunt admittances and off-nominal taps: every
    bus phase gets g^sh U[0, g_max] and b^sh U[-b_max, b_max] (p.u.), every
    line phase gets from- and to-side g^s U[0, g_max], b^s U[0, b_max] (line
    charging) and a squared-voltage tap ratio tau U[1 - tap_dev, 1 + tap_dev].
    Phases a bus or line does not have keep zeros and tau = 1."""
    rng = np.random.default_rng(seed)
    f = dict(feeder)
    nb, nl = int(feeder["n_bus"]), len(feeder["line_from"])

    def masked(mask_arr, n, lo, hi, fill):
        v = rng.uniform(lo, hi, size=(n, 3))
        on = np.array([[(int(m) >> p) & 1 for p in range(3)] for m in mask_arr], dtype=bool)
        return np.where(on, v, fill)

    f["bus_gsh"] = masked(feeder["bus_phases"], nb, 0.0, g_max, 0.0)
    f["bus_bsh"] = masked(feeder["bus_phases"], nb, -b_max, b_max, 0.0)
    f["line_gs_from"] = masked(feeder["line_phases"], nl, 0.0, g_max, 0.0)
    f["line_bs_from"] = masked(feeder["line_phases"], nl, 0.0, b_max, 0.0)
    f["line_gs_to"] = masked(feeder["line_phases"], nl, 0.0, g_max, 0.0)
    f["line_bs_to"] = masked(feeder["line_phases"], nl, 0.0, b_max, 0.0)
    f["line_tap"] = masked(feeder["line_phases"], nl, 1.0 - tap_dev, 1.0 + tap_dev, 1.0)
    f["meta"] = dict(feeder["meta"], shunt_tap_seed=seed)
    return f


def random_generic(seed: int, n_global=40, n_sub=12, max_n=9, p_free=0.0):
    """Random instance of the consensus LP form (c, bounds, {A_s, b_s, idx_s}).

    Every variable has a finite box unless drawn free (probability
    ``p_free``).  Every global variable appears in at least one subsystem and
    at most once in each; b_s is built from a point inside the bounds so each local system is
    consistent.  Some A_s get a duplicated (scaled) row so that rank deficiency
    is exercised.
    """
    rng = np.random.default_rng(seed)
    free = rng.random(n_global) < p_free
    lb = np.where(free, -np.inf, rng.uniform(-2, 0, n_global))
    ub = np.where(free, np.inf, rng.uniform(0.5, 2, n_global))
    xf = np.clip(rng.uniform(-0.4, 0.4, n_global), lb, ub)
    c = rng.uniform(-1, 1, n_global)
    members = [set(rng.choice(n_global, size=int(rng.integers(2, max_n + 1)), replace=False).tolist())
               for _ in range(n_sub)]
    for i in range(n_global):
        if not any(i in m for m in members):
            members[int(rng.integers(n_sub))].add(i)
    subs = []
    for m in members:
        idx = np.array(sorted(m), dtype=np.int32)
        n_s = len(idx)
        m_s = int(rng.integers(1, n_s))
        A = rng.normal(size=(m_s, n_s))
        if m_s >= 2 and rng.random() < 0.3:
            A[-1] = 2.0 * A[0]
        subs.append({"idx": idx, "A": A, "b": A @ xf[idx]})
    return {"c": c, "lb": lb, "ub": ub, "subs": subs}
