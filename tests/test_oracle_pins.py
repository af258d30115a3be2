"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test reaches the same
quantity by a different route (phasor physics, an exact AC power flow, KKT
solves, brute-force minimisation, two independent LP solvers, the paper's
printed counts).
"""
import math

import numpy as np
import pytest

from paper_2310_09410_gb300 import synth
from oracle import admm, lindist

SQ3 = math.sqrt(3.0)
THETA = np.array([0.0, -2 * math.pi / 3, 2 * math.pi / 3])   # phase angles a, b, c


def two_bus(z_r, z_x, ph=7, load=None, alpha=0.0, beta=0.0, delta=False):
    """Root bus 0 (w = 1) feeding bus 1 through one line, one load at bus 1."""
    f = {
        "n_bus": 2,
        "bus_phases": np.array([7, ph], dtype=np.uint8),
        "bus_wmin": np.array([[1.0] * 3, [0.5] * 3]),
        "bus_wmax": np.array([[1.0] * 3, [1.5] * 3]),
        "bus_gsh": np.zeros((2, 3)), "bus_bsh": np.zeros((2, 3)),
        "line_from": np.array([0], dtype=np.int32), "line_to": np.array([1], dtype=np.int32),
        "line_phases": np.array([ph], dtype=np.uint8),
        "line_r": np.array([z_r]), "line_x": np.array([z_x]),
        "line_gs_from": np.zeros((1, 3)), "line_bs_from": np.zeros((1, 3)),
        "line_gs_to": np.zeros((1, 3)), "line_bs_to": np.zeros((1, 3)),
        "line_tap": np.ones((1, 3)),
        "load_bus": np.array([1], dtype=np.int32), "load_phases": np.array([ph], dtype=np.uint8),
        "load_delta": np.array([1 if delta else 0], dtype=np.uint8),
        "load_a": np.array([load.real]), "load_b": np.array([load.imag]),
        "load_alpha": np.full((1, 3), alpha), "load_beta": np.full((1, 3), beta),
        "gen_bus": np.array([0], dtype=np.int32), "gen_phases": np.array([7], dtype=np.uint8),
        "gen_pmin": np.full((1, 3), -np.inf), "gen_pmax": np.full((1, 3), np.inf),
        "gen_qmin": np.full((1, 3), -np.inf), "gen_qmax": np.full((1, 3), np.inf),
        "gen_cost": np.array([1.0]),
    }
    return f


def rand_z(rng, scale):
    r = rng.uniform(0.1, 0.6, size=(3, 3))
    x = rng.uniform(0.1, 0.6, size=(3, 3))
    r, x = 0.5 * (r + r.T) * scale, 0.5 * (x + x.T) * scale
    return r, x


# --- Sec. II-A: linearized line flow -------------------------------------

def test_mp_mq_match_phasor_linearization():
    """M^p, M^q equal the first-order expansion of |V_j|^2 = |V_i - Z I|^2 with
    balanced 120-degree phase angles: each entry is -2 Re(conj(z) e^{j(th_p - th_q)} s)
    for a unit active (s = 1) or reactive (s = j) flow on phase q."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        r, x = rand_z(rng, 1.0)
        mp, mq = lindist.mp_mq(r, x)
        z = r + 1j * x
        for p in range(3):
            for q in range(3):
                g = np.exp(1j * (THETA[p] - THETA[q]))
                assert mp[p, q] == pytest.approx(-2 * (np.conj(z[p, q]) * g * 1.0).real, abs=1e-12)
                assert mq[p, q] == pytest.approx(-2 * (np.conj(z[p, q]) * g * 1j).real, abs=1e-12)


def test_single_phase_and_balanced_reduce_to_distflow():
    """Single phase: w_j = w_i - 2(rP + xQ).  Balanced three-phase flow on a
    line with equal mutuals: the positive-sequence drop 2((r_s - r_m)P + (x_s - x_m)Q)."""
    r = np.array([[0.3, 0.1, 0.1], [0.1, 0.3, 0.1], [0.1, 0.1, 0.3]])
    x = np.array([[0.5, 0.2, 0.2], [0.2, 0.5, 0.2], [0.2, 0.2, 0.5]])
    mp, mq = lindist.mp_mq(r, x)
    P, Q = 0.7, 0.4
    drop = -(mp @ np.full(3, P) + mq @ np.full(3, Q))     # w_i - w_j
    assert np.allclose(drop, 2 * ((0.3 - 0.1) * P + (0.5 - 0.2) * Q))
    assert mp[1, 1] == -2 * r[1, 1] and mq[2, 2] == -2 * x[2, 2]


def ac_power_flow(z, s_load, ph):
    """Exact unbalanced AC power flow, source bus at 1 p.u. with 120-degree
    angles, one line, constant-power load: fixed point V1 = V0 - Z conj(S/V1)."""
    idx = [p for p in range(3) if (ph >> p) & 1]
    v0 = np.exp(1j * THETA[idx])
    zz = z[np.ix_(idx, idx)]
    s = s_load[idx]
    v1 = v0.copy()
    for _ in range(200):
        i = np.conj(s / v1)
        v1 = v0 - zz @ i
    w = np.ones(3)
    w[idx] = np.abs(v1) ** 2
    return w


@pytest.mark.parametrize("ph", [7, 3, 6, 1, 4])
def test_lp_matches_exact_ac_flow_to_first_order(ph):
    """The LP's bus-1 voltage approaches the exact AC solution quadratically in
    the load: dividing the load by 10 cuts the error about 100x."""
    rng = np.random.default_rng(100 + ph)
    r, x = rand_z(rng, 0.05)
    s = rng.uniform(0.2, 1.0, 3) + 1j * rng.uniform(0.05, 0.4, 3)
    errs, drops = [], []
    for scale in (0.1, 0.01):
        sl = s * scale
        f = two_bus(r, x, ph=ph, load=sl)
        M = lindist.build(f)
        obj, xs = admm.lp_optimum(M)
        w_ac = ac_power_flow(r + 1j * x, sl, ph)
        wv = [k for k, nm in enumerate(M.names) if nm[0] == "bus" and nm[1] == 1]
        w_lp = xs[wv]
        w_ex = np.array([w_ac[nm[2]] for nm in (M.names[k] for k in wv)])
        errs.append(np.max(np.abs(w_lp - w_ex)))
        drops.append(np.max(np.abs(1 - w_ex)))
        # lossless model: the source supplies exactly the load
        on = [p for p in range(3) if (ph >> p) & 1]
        assert obj == pytest.approx(float(np.sum(sl.real[on])), rel=1e-9)
    assert errs[1] < drops[1] * 0.05
    assert errs[1] < errs[0] / 50.0


def chain_feeder(zs, ph, loads, ysh, yi, yj, tau):
    """Buses 0 - 1 - ... - n-1 in a chain, every line on phase set ``ph``;
    bus 0 is the source (w = 1), bus k >= 1 has load loads[k-1] (complex, per
    phase) and shunt ysh[k-1] = g^sh + j b^sh; line k has impedance zs[k],
    from-side and to-side shunts yi[k], yj[k] = g^s + j b^s and squared-voltage
    tap ratio tau[k] (per phase)."""
    n = len(zs) + 1
    f = two_bus(zs[0].real, zs[0].imag, ph=ph, load=loads[0])
    f.update({
        "n_bus": n,
        "bus_phases": np.array([7] + [ph] * (n - 1), dtype=np.uint8),
        "bus_wmin": np.array([[1.0] * 3] + [[0.5] * 3] * (n - 1)),
        "bus_wmax": np.array([[1.0] * 3] + [[1.5] * 3] * (n - 1)),
        "bus_gsh": np.vstack([np.zeros(3)] + [y.real for y in ysh]),
        "bus_bsh": np.vstack([np.zeros(3)] + [y.imag for y in ysh]),
        "line_from": np.arange(n - 1, dtype=np.int32), "line_to": np.arange(1, n, dtype=np.int32),
        "line_phases": np.full(n - 1, ph, dtype=np.uint8),
        "line_r": np.array([z.real for z in zs]), "line_x": np.array([z.imag for z in zs]),
        "line_gs_from": np.array([y.real for y in yi]), "line_bs_from": np.array([y.imag for y in yi]),
        "line_gs_to": np.array([y.real for y in yj]), "line_bs_to": np.array([y.imag for y in yj]),
        "line_tap": np.array(tau),
        "load_bus": np.arange(1, n, dtype=np.int32), "load_phases": np.full(n - 1, ph, dtype=np.uint8),
        "load_delta": np.zeros(n - 1, dtype=np.uint8),
        "load_a": np.array([l.real for l in loads]), "load_b": np.array([l.imag for l in loads]),
        "load_alpha": np.zeros((n - 1, 3)), "load_beta": np.zeros((n - 1, 3)),
    })
    return f


def ac_chain_flow(zs, ph, loads, ysh, yi, yj, tau, sweeps=400):
    """Exact unbalanced AC power flow of the chain: each line is a pi model
    (shunt yi at the from end, series impedance Z, an ideal transformer whose
    primary voltage is sqrt(tau) times the secondary's, shunt yj at the to
    end); a shunt admittance y at squared voltage w draws w conj(y); loads
    have constant power.  Backward/forward sweeps from a flat start.
    Returns w per bus and the complex power entering each line at its from
    end (S_ij) and at its to end (S_ji), on the phases of ``ph``."""
    idx = [p for p in range(3) if (ph >> p) & 1]
    n = len(zs) + 1
    t = [np.sqrt(np.asarray(tk)[idx]) for tk in tau]
    v = [np.exp(1j * THETA[idx])]
    for k in range(n - 1):
        v.append(v[-1] / t[k])
    for _ in range(sweeps):
        s_into = None                     # power bus k+1 sends into line k+1
        ip, s_ij, s_ji = [None] * (n - 1), [None] * (n - 1), [None] * (n - 1)
        for k in range(n - 2, -1, -1):
            j = k + 1
            wj = np.abs(v[j]) ** 2
            s_del = loads[j - 1][idx] + wj * np.conj(ysh[j - 1][idx]) + (0 if s_into is None else s_into)
            s_t = s_del + wj * np.conj(yj[k][idx])
            ip[k] = np.conj(s_t / v[j]) / t[k]
            s_ji[k] = -s_del
            s_ij[k] = v[k] * np.conj(ip[k]) + np.abs(v[k]) ** 2 * np.conj(yi[k][idx])
            s_into = s_ij[k]
        for k in range(n - 1):
            zz = zs[k][np.ix_(idx, idx)]
            v[k + 1] = (v[k] - zz @ ip[k]) / t[k]
    w = [np.abs(vk) ** 2 for vk in v]
    return w, s_ij, s_ji


def chain_case(rng, ph, n_lines=2):
    zs, loads, ysh, yi, yj, tau = [], [], [], [], [], []
    for _ in range(n_lines):
        r, x = rand_z(rng, 0.05)
        zs.append(r + 1j * x)
        loads.append(rng.uniform(0.2, 1.0, 3) + 1j * rng.uniform(0.05, 0.4, 3))
        ysh.append(rng.uniform(0.05, 0.3, 3) + 1j * rng.uniform(-0.4, 0.4, 3))
        yi.append(rng.uniform(0.05, 0.3, 3) + 1j * rng.uniform(0.1, 0.5, 3))
        yj.append(rng.uniform(0.05, 0.3, 3) + 1j * rng.uniform(0.1, 0.5, 3))
        # one tap per line on multi-phase lines: the model's drop term takes the
        # phase voltages as balanced in magnitude, which unequal taps break at
        # first order; per-phase values where one phase is on
        tau.append(rng.uniform(0.95, 1.05, 3) if ph in (1, 2, 4) else np.full(3, rng.uniform(0.95, 1.05)))
    return zs, loads, ysh, yi, yj, tau


def chain_errors(ph, seed):
    """LP optimum of the chain against the exact AC flow with loads and
    shunts scaled by 0.1 and 0.01 (taps fixed): max errors of w, line flows
    and objective at each scale, and the size of the first-order effects
    (the voltage deviation from the no-load profile and the largest flow)."""
    rng = np.random.default_rng(seed)
    zs, loads, ysh, yi, yj, tau = chain_case(rng, ph)
    idx = [p for p in range(3) if (ph >> p) & 1]
    out = []
    for scale in (0.1, 0.01):
        sc = [[y * scale for y in arr] for arr in (loads, ysh, yi, yj)]
        f = chain_feeder(zs, ph, sc[0], sc[1], sc[2], sc[3], tau)
        M = lindist.build(f)
        obj, xs = admm.lp_optimum(M)
        w_ex, s_ij, s_ji = ac_chain_flow(zs, ph, sc[0], sc[1], sc[2], sc[3], tau)
        w0 = [np.ones(len(idx))]
        for k in range(len(zs)):
            w0.append(w0[-1] / np.asarray(tau[k])[idx])      # no-load profile
        ew, ef, dev, big = 0.0, 0.0, 0.0, 0.0
        for k, nm in enumerate(M.names):
            if nm[0] == "bus" and nm[1] >= 1:
                pos = idx.index(nm[2])
                ew = max(ew, abs(xs[k] - w_ex[nm[1]][pos]))
                dev = max(dev, abs(w_ex[nm[1]][pos] - w0[nm[1]][pos]))
            if nm[0] == "line":
                pos = idx.index(nm[2])
                ex = {"pij": s_ij[nm[1]].real, "qij": s_ij[nm[1]].imag,
                      "pji": s_ji[nm[1]].real, "qji": s_ji[nm[1]].imag}[nm[3]][pos]
                ef = max(ef, abs(xs[k] - ex))
                big = max(big, abs(ex))
        eo = abs(obj - float(np.sum(s_ij[0].real)))
        out.append((ew, ef, eo, dev, big))
    return out


def chain_pin_holds(errs):
    (w1, f1, o1, _, _), (w2, f2, o2, dev2, big2) = errs
    quadratic = w2 < w1 / 50.0 and f2 < f1 / 50.0 and o2 < o1 / 50.0
    small = w2 < 0.05 * dev2 and f2 < 0.05 * big2
    return quadratic and small


@pytest.mark.parametrize("ph", [7, 3, 6, 1, 2, 4])
def test_shunts_and_taps_match_exact_ac_flow_to_first_order(ph):
    """Eq. balance_eqns (g^sh, b^sh) and Eq. power_flow_eqns (g^s, b^s at both
    ends, tap tau): on a three-bus chain (a bus subsystem with loads, shunts
    and two lines, a line subsystem, a leaf) the LP's voltages, line flows
    and objective approach the exact pi-model AC power flow quadratically as
    the loads and shunt admittances shrink, with off-nominal taps held."""
    assert chain_pin_holds(chain_errors(ph, 200 + ph))


MUTATIONS = {
    # a sign error in one shunt term, or the tap on the wrong side of the line
    "bus g^sh sign": ("_bus_rows", lambda f: dict(f, bus_gsh=-f["bus_gsh"])),
    "bus b^sh sign": ("_bus_rows", lambda f: dict(f, bus_bsh=-f["bus_bsh"])),
    "from g^s sign": ("_line_rows", lambda f: dict(f, line_gs_from=-f["line_gs_from"])),
    "from b^s sign": ("_line_rows", lambda f: dict(f, line_bs_from=-f["line_bs_from"])),
    "to g^s sign": ("_line_rows", lambda f: dict(f, line_gs_to=-f["line_gs_to"])),
    "to b^s sign": ("_line_rows", lambda f: dict(f, line_bs_to=-f["line_bs_to"])),
    "tap inverted": ("_line_rows", lambda f: dict(f, line_tap=1.0 / f["line_tap"])),
}


@pytest.mark.parametrize("mutation", sorted(MUTATIONS))
def test_shunt_tap_pin_catches_planted_errors(monkeypatch, mutation):
    """The pin above fails when one shunt or tap term of the oracle's rows is
    planted with a plausible mistake."""
    fn, change = MUTATIONS[mutation]
    orig = getattr(lindist, fn)
    monkeypatch.setattr(lindist, fn, lambda f, *a, **k: orig(change(f), *a, **k))
    assert not chain_pin_holds(chain_errors(7, 207))


# --- Sec. II-A: load model -----------------------------------------------

@pytest.mark.parametrize("alpha", [0.0, 1.0, 2.0])
def test_vdlm_is_first_order_zip(alpha):
    """VDLM-1 is the tangent at w = 1 of the ZIP law p = a w^(alpha/2):
    constant power, current, impedance for alpha = 0, 1, 2."""
    a = 0.37
    f = two_bus(np.eye(3) * 1e-3, np.eye(3) * 1e-3, ph=1, load=np.array([a + 0.1j, 0, 0]), alpha=alpha)
    M = lindist.build(f)
    leaf = [s for s in M.subs if s["kind"] == "leaf"][0]
    pd = [k for k, g in enumerate(leaf["idx"]) if M.names[g][3] == "pd"][0]
    w = [k for k, g in enumerate(leaf["idx"]) if M.names[g][0] == "bus" and M.names[g][1] == 1][0]
    row = [r for r in range(leaf["A"].shape[0]) if leaf["A"][r, pd] != 0 and leaf["A"][r].nonzero()[0].size <= 2][0]
    for wv in (1.0 + 1e-3, 1.0 - 2e-3):
        # solve the row for p^d at this w
        coef = leaf["A"][row]
        pd_val = (leaf["b"][row] - coef[w] * wv) / coef[pd]
        exact = a * wv ** (alpha / 2)
        assert abs(pd_val - exact) <= 2 * a * (wv - 1) ** 2 + 1e-15


def test_delta_rows_match_phasor_currents():
    """VDLM-6..10 hold for the bus-side powers of delta branch loads computed
    from phasors: branch ab, bc, ca carrying S_d draws V_p conj(I) at its ends
    with I = conj(S_d / V_branch)."""
    rng = np.random.default_rng(3)
    v = np.exp(1j * THETA)
    for _ in range(5):
        sd = rng.uniform(0.1, 1, 3) + 1j * rng.uniform(0.0, 0.5, 3)
        sb = np.zeros(3, dtype=complex)
        for k, (p, q) in enumerate([(0, 1), (1, 2), (2, 0)]):
            i = np.conj(sd[k] / (v[p] - v[q]))
            sb[p] += v[p] * np.conj(i)
            sb[q] -= v[q] * np.conj(i)
        f = two_bus(np.eye(3) * 1e-3, np.eye(3) * 1e-3, ph=7, load=sd, delta=True)
        M = lindist.build(f)
        leaf = [s for s in M.subs if s["kind"] == "leaf"][0]
        val = {}
        for k, g in enumerate(leaf["idx"]):
            nm = M.names[g]
            if nm[0] == "load":
                val[k] = {"pb": sb[nm[2]].real, "qb": sb[nm[2]].imag,
                          "pd": sd[nm[2]].real, "qd": sd[nm[2]].imag}[nm[3]]
        load_cols = sorted(val)
        for r in range(leaf["A"].shape[0]):
            row = leaf["A"][r]
            if np.all(row[[k for k in range(len(row)) if k not in val]] == 0):
                lhs = sum(row[k] * val[k] for k in load_cols)
                if any(row[k] != 0 and M.names[leaf["idx"][k]][3] == "pb" for k in load_cols):
                    assert lhs == pytest.approx(leaf["b"][r], abs=1e-12)


# --- Sec. V-A decomposition ------------------------------------------------

def test_table3_counts_follow_merge_rule():
    """Table III prints nodes, lines, leaves and S for the four IEEE feeders;
    merging each leaf into its line gives S = nodes + lines - leaves."""
    rows = np.loadtxt(__file__.replace("test_oracle_pins.py", "golden/table3_subsystems.txt"), comments="#")
    for nodes, lines, leaves, S in rows:
        assert nodes + lines - leaves == S


@pytest.mark.parametrize("name,seed", [("13", 1001), ("34", 5034), ("123", 2001), ("8500", 3001)])
def test_decomposition_structure(name, seed):
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    nb = f["n_bus"]
    assert len(M.subs) == nb + (nb - 1) - M.leaves
    counts = np.bincount(np.concatenate([s["idx"] for s in M.subs]), minlength=M.n)
    assert counts.min() >= 1                               # every variable has a copy
    for s in M.subs:
        assert len(np.unique(s["idx"])) == len(s["idx"])   # B_s: one 1 per column at most
    A, b = lindist.centralized(M)
    assert A.shape == (sum(s["A"].shape[0] for s in M.subs), M.n)
    # lossless, shunt-free: every equation set is full row rank
    if M.n < 3000:
        assert np.linalg.matrix_rank(A) == A.shape[0]


# --- Sec. III-B closed forms -------------------------------------------------

def subsystems_for_pins():
    out = []
    M = lindist.build(synth.preset_feeder("13", 1001))
    out += [(s["A"], s["b"]) for s in M.subs]
    g = synth.random_generic(5)
    out += [(s["A"], s["b"]) for s in g["subs"]]
    return out


def test_closed_form_projection_algebra():
    """-Abar is the orthogonal projector onto null(A_s); bbar solves A_s x = b_s
    and lies in row(A_s)."""
    for A, b in subsystems_for_pins():
        Ab, bb = admm.precompute(A, b)
        Mproj = -Ab
        n = A.shape[1]
        assert np.allclose(Mproj, Mproj.T, atol=1e-12)
        assert np.allclose(Mproj @ Mproj, Mproj, atol=1e-11)
        assert np.allclose(A @ Mproj, 0, atol=1e-11 * max(1, np.abs(A).max()))
        assert np.allclose(A @ bb, b, atol=1e-11 * max(1, np.abs(b).max()))
        assert np.allclose(Mproj @ bb, 0, atol=1e-11)
        assert np.trace(Mproj) == pytest.approx(n - np.linalg.matrix_rank(A), abs=1e-9)


def test_local_update_equals_kkt_solution():
    """x_s of Eq. closed_2 equals the solution of the KKT system of ADMM-2,
    [rho I  A^T; A 0][x; mu] = [rho v + lam; b], solved by dense LU."""
    rng = np.random.default_rng(11)
    rho = 100.0
    for A, b in subsystems_for_pins():
        Ab, bb = admm.precompute(A, b)
        n = A.shape[1]
        bx = rng.normal(size=n)       # B_s x
        lam = rng.normal(size=n) * 10
        d = -rho * bx - lam
        x_closed = Ab @ d / rho + bb
        # independent rows only (the dense KKT matrix must be nonsingular)
        q, r, piv = __import__("scipy.linalg", fromlist=["qr"]).qr(A.T, pivoting=True)
        rank = int(np.sum(np.abs(np.diag(r)) > 1e-12 * max(1, np.linalg.norm(A))))
        keep = np.sort(piv[:rank])
        Ar, br = A[keep], b[keep]
        K = np.block([[rho * np.eye(n), Ar.T], [Ar, np.zeros((rank, rank))]])
        sol = np.linalg.solve(K, np.concatenate([rho * bx + lam, br]))
        assert np.allclose(x_closed, sol[:n], atol=1e-10)


def test_inconsistent_local_system_rejected():
    A = np.array([[1.0, 2.0, 0.0], [2.0, 4.0, 0.0]])
    with pytest.raises(ValueError):
        admm.precompute(A, np.array([1.0, 3.0]))


# --- Algorithm 1, one iteration against brute force ----------------------

def test_first_iteration_against_bruteforce():
    """From an arbitrary state (x_s, lam): the global step minimises the full
    ADMM-1 objective over the box (checked by bounded L-BFGS), then the local
    step solves ADMM-2 (checked by a KKT solve) and lam follows ADMM-3."""
    from scipy.optimize import minimize
    g = synth.random_generic(21, n_global=15, n_sub=6, max_n=6)
    M = lindist.from_generic(g)
    P = admm.Prepared(M)
    rng = np.random.default_rng(0)
    L = len(P.gidx)
    xs0 = rng.normal(size=L)
    lam0 = rng.normal(size=L) * 30
    rho = 7.0
    r = admm.admm(P, rho=rho, max_iter=1, check_every=0, xs=xs0, lam=lam0)

    def f(x):
        return M.c @ x + lam0 @ x[P.gidx] + 0.5 * rho * np.sum((x[P.gidx] - xs0) ** 2)

    def grad(x):
        gr = M.c.copy()
        np.add.at(gr, P.gidx, lam0 + rho * (x[P.gidx] - xs0))
        return gr
    res = minimize(f, np.clip(np.zeros(M.n), M.lb, M.ub), jac=grad, method="L-BFGS-B",
                   bounds=list(zip(M.lb, M.ub)), options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    assert np.allclose(r.x, res.x, atol=1e-6)
    assert f(r.x) <= f(res.x) + 1e-9
    # per-variable ternary search of the 1-D problem
    for i in range(M.n):
        ks = np.flatnonzero(P.gidx == i)
        lo, hi = max(M.lb[i], -50), min(M.ub[i], 50)
        h = lambda t: (M.c[i] + lam0[ks].sum()) * t + 0.5 * rho * np.sum((t - xs0[ks]) ** 2)
        for _ in range(200):
            a, b_ = lo + (hi - lo) / 3, hi - (hi - lo) / 3
            lo, hi = (a, hi) if h(a) > h(b_) else (lo, b_)
        assert r.x[i] == pytest.approx(0.5 * (lo + hi), abs=1e-7)   # ternary search resolves ~sqrt(eps)
    # local step = ADMM-2 optimum, dual = ADMM-3
    for si, s in enumerate(M.subs):
        sl = slice(P.off[si], P.off[si + 1])
        A, b = s["A"], s["b"]
        from scipy.optimize import minimize as mn
        n = len(s["idx"])
        bx = r.x[s["idx"]]
        obj = lambda y: -lam0[sl] @ y + 0.5 * rho * np.sum((bx - y) ** 2)
        cons = {"type": "eq", "fun": lambda y: A @ y - b, "jac": lambda y: A}
        sol = mn(obj, bx, jac=lambda y: -lam0[sl] - rho * (bx - y), constraints=[cons], method="SLSQP",
                 options={"ftol": 1e-14, "maxiter": 500})
        assert np.allclose(r.xs[sl], sol.x, atol=1e-6)
        assert np.allclose(r.lam[sl], lam0[sl] + rho * (bx - r.xs[sl]), atol=1e-9)


# --- convergence to the centralized LP (Eq. LP_model) ---------------------

@pytest.mark.parametrize("seed", [1001, 1002])
def test_lp_solvers_agree_and_admm_converges(seed):
    M = lindist.build(synth.preset_feeder("13", seed))
    obj_h, _ = admm.lp_optimum(M)
    A, b = lindist.centralized(M)
    obj_i, _ = admm.dense_ipm(M.c, A, b, M.lb, M.ub)
    assert obj_i == pytest.approx(obj_h, rel=1e-10)
    r = admm.admm(M, eps_rel=1e-10, max_iter=20000)
    assert r.converged
    assert r.objective == pytest.approx(obj_h, rel=1e-8)


def test_stopping_rule_meets_objective_bar():
    """At eps_rel = 1e-8 (with pres <= 1e-4) the objective is within 1e-6."""
    for name, seed in (("13", 1003), ("34", 5034)):
        M = lindist.build(synth.preset_feeder(name, seed))
        obj, _ = admm.lp_optimum(M)
        r = admm.admm(M, eps_rel=1e-8, eps_abs_pres=1e-4, max_iter=60000)
        assert r.converged and r.pres <= 1e-4
        assert abs(r.objective - obj) <= 1e-6 * abs(obj)


def test_generic_instances_converge():
    # random consensus LPs; plain ADMM is slow on some draws, these converge
    # within a few thousand iterations
    for seed in (1, 7, 8, 13, 14):
        M = lindist.from_generic(synth.random_generic(seed))
        obj, _ = admm.lp_optimum(M)
        r = admm.admm(M, rho=1.0, eps_rel=1e-10, eps_abs_pres=1e-8, max_iter=20000)
        assert r.converged
        assert r.objective == pytest.approx(obj, rel=1e-7, abs=1e-8)


def test_single_subsystem_is_centralized_lp():
    """S = 1 (Sec. I): one subsystem holding every row, B = I."""
    M = lindist.build(synth.preset_feeder("13", 1004))
    A, b = lindist.centralized(M)
    M1 = lindist.Model()
    M1.n, M1.c, M1.lb, M1.ub, M1.is_voltage, M1.names = M.n, M.c, M.lb, M.ub, M.is_voltage, M.names
    M1.subs = [{"kind": "all", "owner": 0, "idx": np.arange(M.n), "A": A, "b": b}]
    obj, _ = admm.lp_optimum(M)
    r = admm.admm(M1, eps_rel=1e-10, max_iter=50000)
    assert r.converged
    assert r.objective == pytest.approx(obj, rel=1e-8)


def test_kkt_at_convergence():
    """Consensus, the linearized power-flow equalities, bounds, lam_s in
    row(A_s) and the sign of the reduced cost c_i + sum lam_k."""
    M = lindist.build(synth.preset_feeder("13", 1001))
    P = admm.Prepared(M)
    r = admm.admm(P, eps_rel=1e-12, eps_abs_pres=1e-10, max_iter=30000)
    assert r.converged
    xg = r.x[P.gidx]
    assert np.linalg.norm(xg - r.xs) <= 1e-9
    for si, s in enumerate(M.subs):
        sl = slice(P.off[si], P.off[si + 1])
        assert np.allclose(s["A"] @ r.x[s["idx"]], s["b"], atol=1e-8)
        Ab, _ = admm.precompute(s["A"], s["b"])
        assert np.allclose(Ab @ r.lam[sl], 0, atol=1e-6)
    assert np.all(r.x >= M.lb - 1e-15) and np.all(r.x <= M.ub + 1e-15)
    red = M.c.copy()
    np.add.at(red, P.gidx, r.lam)
    tol = 1e-5 * max(1.0, np.abs(M.c).max())
    at_lb = np.abs(r.x - M.lb) <= 1e-9
    at_ub = np.abs(r.x - M.ub) <= 1e-9
    interior = ~at_lb & ~at_ub
    assert np.all(np.abs(red[interior]) <= tol)
    assert np.all(red[at_lb & ~at_ub] >= -tol)
    assert np.all(red[at_ub & ~at_lb] <= tol)
    # lossless: generation equals demand
    pg = sum(r.x[k] for k, nm in enumerate(M.names) if nm[0] == "gen" and nm[3] == "p")
    pd = sum(r.x[k] for k, nm in enumerate(M.names) if nm[0] == "load" and nm[3] == "pd")
    assert pg == pytest.approx(pd, abs=1e-8)


def test_init_point_rule():
    M = lindist.build(synth.preset_feeder("13", 1001))
    x0 = admm.init_point(M)
    for k, nm in enumerate(M.names):
        if nm[0] == "bus":
            assert x0[k] == 1.0
        elif nm[0] == "gen" and nm[1] > 0:
            assert x0[k] == pytest.approx(0.5 * (M.lb[k] + M.ub[k]))
        elif nm[0] in ("load", "line") or (nm[0] == "gen" and nm[1] == 0):
            assert x0[k] == 0.0


# --- Sec. III-C quantities against the iterates ---------------------------

def test_residual_history_matches_the_iterates():
    """The quantities the oracle records after iteration t + 1, against the
    states of separate runs of t and t + 1 iterations: pres equals
    |lambda^{t+1} - lambda^t| / rho (the dual update, Eq. ADMM-3), dres is rho
    |x_s^{t+1} - x_s^t|, the norms behind eps_prim and eps_dual are those of
    B x^{t+1}, x_s^{t+1} and lambda^{t+1}, and the objective is c^T x^{t+1}
    (an off-by-one in the oracle's bookkeeping of the previous state fails)."""
    M = lindist.build(synth.preset_feeder("13", 1001))
    P = admm.Prepared(M)
    rho = 100.0
    rec = admm.admm(P, rho=rho, max_iter=40, check_every=0, record=True)
    for t in (0, 1, 9, 39):
        if t == 0:
            lam_t, xs_t = np.zeros(len(P.gidx)), P.x0[P.gidx]
        else:
            a = admm.admm(P, rho=rho, max_iter=t, check_every=0)
            lam_t, xs_t = a.lam, a.xs
        b = admm.admm(P, rho=rho, max_iter=t + 1, check_every=0)
        pres, dres, eprim, edual, obj = rec.hist[t]
        assert pres == pytest.approx(np.linalg.norm(b.lam - lam_t) / rho, rel=1e-9)
        assert pres == pytest.approx(np.linalg.norm(b.x[P.gidx] - b.xs), rel=1e-12)
        assert dres == pytest.approx(rho * np.linalg.norm(b.xs - xs_t), rel=1e-12)
        assert eprim == pytest.approx(max(np.linalg.norm(b.x[P.gidx]), np.linalg.norm(b.xs)), rel=1e-12)
        assert edual == pytest.approx(np.linalg.norm(b.lam), rel=1e-12)
        assert obj == pytest.approx(M.c @ b.x, rel=1e-12)
