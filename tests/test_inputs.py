"""The seeded synthetic feeders and load scenarios against the workload recipe
they stand in for (the 13-, 123- and 8500-bus configurations and the batch
of load scenarios): sizes, tree shape, phase sets, line, load and generator
data, bounds, costs and scenario factors.  CPU only."""
import math

import numpy as np
import pytest

from paper_2310_09410_gb300 import synth

ALLOWED = {7, 3, 6, 1, 2, 4}          # abc, ab, bc, a, b, c ("ac" excluded)
SINGLE = {1, 2, 4}


def phases(mask):
    return [p for p in range(3) if (int(mask) >> p) & 1]


CASES = [("13", 1001, 13, 9, 2, 6, None), ("13", 1002, 13, 9, 2, 6, None),
         ("34", 5034, 34, 24, 4, 12, None), ("123", 2001, 123, 85, 10, 30, 0.4),
         ("8500", 3001, 8500, 1200, 100, 60, 0.7)]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] + "-" + str(c[1]) for c in CASES])
def case(request):
    name, seed, n_bus, n_load, n_der, dmax, p1 = request.param
    return synth.preset_feeder(name, seed), n_bus, n_load, n_der, dmax, p1


def test_radial_tree_and_depth(case):
    f, n_bus, _, _, dmax, _ = case
    assert f["n_bus"] == n_bus
    assert len(f["line_from"]) == n_bus - 1
    assert np.array_equal(f["line_to"], np.arange(1, n_bus))
    assert np.all(f["line_from"] < f["line_to"])          # a parent precedes its child
    depth = np.zeros(n_bus, dtype=int)
    for e in range(n_bus - 1):
        depth[f["line_to"][e]] = depth[f["line_from"][e]] + 1
    assert depth.max() <= dmax and depth.max() == f["meta"]["depth"]


def test_phase_sets_nested(case):
    f, n_bus, _, _, _, p1 = case
    bus_ph = f["bus_phases"]
    assert bus_ph[0] == 7
    for e in range(n_bus - 1):
        m, par = int(f["line_phases"][e]), int(bus_ph[f["line_from"][e]])
        assert m in ALLOWED
        assert m & ~par == 0                                # a subset of the parent's phases
        assert bus_ph[f["line_to"][e]] == m                 # the bus takes its feeding line's phases
        if f["line_from"][e] == 0:
            assert m == 7                                   # lines leaving the substation are abc
    if p1 is not None:
        frac = float(np.mean([int(m) in SINGLE for m in f["line_phases"]]))
        assert abs(frac - p1) <= 0.05, frac


def test_line_impedances(case):
    f, n_bus, _, _, _, _ = case
    kappa = f["meta"]["kappa"]
    assert kappa > 0
    for e in range(n_bus - 1):
        ph = phases(f["line_phases"][e])
        off = [p for p in range(3) if p not in ph]
        for key in ("line_r", "line_x"):
            z = f[key][e]
            assert np.allclose(z, z.T)
            assert np.all(z[off, :] == 0) and np.all(z[:, off] == 0)
            d = np.diag(z)[ph]
            # diagonals U[0.1, 0.6] ohm/km times one length and one scale
            assert d.min() > 0 and d.max() / d.min() <= 6.0 + 1e-9
            # length U[0.1, 1] km: the diagonal per unit kappa lies in [0.01, 0.6] ohm
            assert np.all(d / kappa >= 0.01 - 1e-12) and np.all(d / kappa <= 0.6 + 1e-12)
            for i, a in enumerate(ph):
                for b in ph[i + 1:]:
                    r = z[a, b] / (0.5 * (z[a, a] + z[b, b]))
                    assert 0.3 - 1e-9 <= r <= 0.5 + 1e-9


def test_loads(case):
    f, n_bus, n_load, _, _, _ = case
    lb = f["load_bus"]
    assert len(lb) == n_load and len(set(lb.tolist())) == n_load and lb.min() >= 1
    assert np.array_equal(f["load_phases"], f["bus_phases"][lb])
    assert not f["load_delta"].any() and not f["load_alpha"].any() and not f["load_beta"].any()
    lo, hi = math.tan(math.acos(0.98)), math.tan(math.acos(0.85))
    for l in range(n_load):
        ph = phases(f["load_phases"][l])
        for p in range(3):
            a, b = f["load_a"][l, p], f["load_b"][l, p]
            if p not in ph:
                assert a == 0 and b == 0
                continue
            assert 0.0 <= a <= 0.200                       # MW per phase (1 MVA per-phase base)
            if a > 0:
                assert lo - 1e-12 <= b / a <= hi + 1e-12   # power factor U[0.85, 0.98]


def test_generators_bounds_costs(case):
    f, n_bus, _, n_der, _, _ = case
    gb = f["gen_bus"]
    assert len(gb) == n_der + 1 and gb[0] == 0
    assert len(set(gb[1:].tolist())) == n_der and gb[1:].min() >= 1
    assert np.all(np.isinf(f["gen_pmax"][0])) and np.all(np.isinf(f["gen_qmin"][0]))
    for g in range(1, n_der + 1):
        ph = phases(f["gen_phases"][g])
        assert int(f["gen_phases"][g]) == int(f["bus_phases"][gb[g]])
        assert np.isclose(f["gen_pmax"][g].sum(), 0.150) and np.all(f["gen_pmin"][g] == 0)
        assert np.isclose(f["gen_qmax"][g].sum(), 0.100) and np.isclose(f["gen_qmin"][g].sum(), -0.100)
        assert np.allclose(f["gen_pmax"][g][ph], 0.150 / len(ph))
    assert np.all((f["gen_cost"] >= 10) & (f["gen_cost"] <= 50))
    assert np.all(f["bus_wmin"][1:] == 0.9025) and np.all(f["bus_wmax"][1:] == 1.1025)
    assert np.all(f["bus_wmin"][0] == 1.0) and np.all(f["bus_wmax"][0] == 1.0)


def test_zero_der_voltage_bound_holds():
    """The impedance scale keeps the conservative zero-DER bound on |w - 1|
    (2 sum over the path of (|r| + |x|)(P + Q) downstream) at 0.068, inside
    the squared-voltage box."""
    f = synth.preset_feeder("123", 2001)
    n = f["n_bus"]
    parent = np.zeros(n, dtype=int)
    parent[f["line_to"]] = f["line_from"]
    down = np.zeros((n, 3))
    for l, b in enumerate(f["load_bus"]):
        down[b] += f["load_a"][l] + f["load_b"][l]
    for k in range(n - 1, 0, -1):
        down[parent[k]] += down[k]
    bound = np.zeros(n)
    for k in range(1, n):
        z = np.abs(f["line_r"][k - 1]) + np.abs(f["line_x"][k - 1])
        bound[k] = bound[parent[k]] + 2.0 * float(np.max(z @ down[k]))
    assert np.isclose(bound.max(), 0.068)
    assert 1.0 - bound.max() > 0.9025


def test_load_scenarios():
    """Scenario j scales every load by U[0.6, 1.2] x N(1, 0.05) (per load),
    drawn from its own seed."""
    f = synth.preset_feeder("123", 2001)
    scales, noise = [], []
    for j in range(200):
        g = synth.load_scenario(f, 4000 + j)
        s = g["meta"]["scenario_scale"]
        scales.append(s)
        active = f["load_a"][:, :] > 0
        fac = g["load_a"][active] / f["load_a"][active]
        per_load = np.array([g["load_a"][l][f["load_a"][l] > 0][0] / f["load_a"][l][f["load_a"][l] > 0][0]
                             for l in range(len(f["load_bus"])) if f["load_a"][l].max() > 0])
        noise.extend((per_load / s).tolist())
        assert np.allclose(g["load_b"][active] / f["load_b"][active], fac)   # P and Q scaled together
    scales = np.array(scales)
    assert scales.min() >= 0.6 and scales.max() <= 1.2
    assert abs(scales.mean() - 0.9) < 0.03
    noise = np.array(noise)
    assert abs(noise.mean() - 1.0) < 0.005 and abs(noise.std() - 0.05) < 0.005
    assert synth.load_scenario(f, 4000)["meta"]["scenario_scale"] == scales[0]   # seeded
