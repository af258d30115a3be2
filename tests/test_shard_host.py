"""Sharded single instance, host side and the multi-rank exchange on CPU.

* opf_partition (host code of the library) assigns every subsystem of a
  feeder to one of n parts, balanced by work, each part a run of subtrees;
* two gloo ranks run Algorithm 1 on the two parts of the 123-bus feeder with
  the exchange the sharded path uses (an all-reduce of the cut globals'
  sigma and of the Sec. III-C sums) and reproduce the unsharded oracle's
  iterates and stopping iteration.  Each rank's local update here is the
  oracle's dense one (the GPU kernels of the shards are covered by
  tests/test_shard_gpu.py); what is under test is the decomposition of the
  global update into partial sums over shards and the exchange protocol.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import admm as oracle_admm, lindist
from paper_2310_09410_gb300 import opf, synth


def part_of(name, seed, n_parts):
    f = synth.preset_feeder(name, seed)
    M = lindist.build(f)
    return f, M, opf.partition(f, n_parts, len(M.subs))


@pytest.mark.parametrize("name,seed,n_parts", [("123", 2001, 2), ("123", 2001, 4), ("8500", 3001, 2),
                                               ("8500", 3001, 8)])
def test_partition_covers_and_balances(name, seed, n_parts):
    f, M, part = part_of(name, seed, n_parts)
    assert part.shape == (len(M.subs),)
    assert set(part.tolist()) == set(range(n_parts))
    work = np.zeros(n_parts)
    for s, p in zip(M.subs, part):
        work[p] += len(s["idx"]) ** 2
    assert work.max() <= 1.25 * work.mean() + 64 ** 2, work
    # the cut: globals with copies on more than one part, a small share
    parts_of = {}
    for s, p in zip(M.subs, part):
        for g in s["idx"]:
            parts_of.setdefault(int(g), set()).add(int(p))
    n_cut = sum(len(v) > 1 for v in parts_of.values())
    assert 0 < n_cut <= 0.05 * M.n + 40, (n_cut, M.n)


def test_partition_parts_are_runs_of_subtrees():
    """In depth-first order every part is one contiguous range, so the buses
    of a part whose parent lies in another part are few."""
    f, M, part = part_of("8500", 3001, 8)
    nb = f["n_bus"]
    parent = np.full(nb, -1)
    parent[f["line_to"]] = f["line_from"]
    has_child = np.zeros(nb, bool)
    has_child[f["line_from"]] = True
    anchors = [i for i in range(nb) if i == 0 or has_child[i]] + list(f["line_to"])
    bus_part = np.full(nb, -1)
    for s, a in enumerate(anchors):
        assert bus_part[a] in (-1, part[s])       # subsystems anchored at one bus share its part
        bus_part[a] = part[s]
    entries = sum(1 for i in range(1, nb) if bus_part[i] != bus_part[parent[i]])
    assert entries <= 8 * 30, entries


def test_partition_rejects_bad_arguments():
    f = synth.preset_feeder("13", 1001)
    with pytest.raises(opf.OPFError):
        opf.partition(f, 2, 3)                   # wrong subsystem count
    with pytest.raises(opf.OPFError):
        opf.partition(f, 0, len(lindist.build(f).subs))


def test_test_rule_matches_its_definition():
    sums = np.array([4e-10, 1e-16, 2.0, 2.1, 9.0, 5.0])
    ok, out = opf.apply_test_rule(sums, rho=100.0, eps_rel=1e-3, eps_abs_pres=1e-4)
    assert ok
    assert out[0] == pytest.approx(2e-5) and out[1] == pytest.approx(1e-6)
    assert out[2] == pytest.approx(np.sqrt(2.1)) and out[3] == pytest.approx(3.0) and out[4] == 5.0
    ok, _ = opf.apply_test_rule(sums, rho=100.0, eps_rel=1e-3, eps_abs_pres=1e-5)
    assert not ok


# ------------------------------------------------------------ two gloo ranks

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _sharded_admm(rank, world, port, out, n_iter, eps_rel):
    """One rank: the subsystems of its part, dense local updates (oracle
    precompute), cut sigma and test sums all-reduced over the ranks."""
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rho = 100.0
        f, M, part = part_of("123", 2001, world)
        P = oracle_admm.Prepared(M)
        mine = [s for s in range(len(M.subs)) if part[s] == rank]
        ntot = np.zeros(M.n)
        parts_of = [set() for _ in range(M.n)]
        for s in range(len(M.subs)):
            for g in M.subs[s]["idx"]:
                ntot[g] += 1
                parts_of[g].add(int(part[s]))
        cut = np.array([g for g in range(M.n) if len(parts_of[g]) > 1])
        owner = np.array([min(p) for p in parts_of])
        blocks = []
        for s in mine:
            o0, o1 = P.off[s], P.off[s + 1]
            n = o1 - o0
            blocks.append((np.arange(o0, o1), P.abar[P.aoff[s]:P.aoff[s] + n * n].reshape(n, n), P.bbar[o0:o1]))
        slots = np.concatenate([b[0] for b in blocks])
        gk = P.gidx[slots]
        xs = P.x0[gk].copy()
        lam = np.zeros(len(slots))
        iters, conv = 0, False
        for t in range(n_iter):
            u = rho * xs - lam
            sigma = np.zeros(M.n)
            np.add.at(sigma, gk, u)
            st = torch.from_numpy(sigma[cut].copy())
            dist.all_reduce(st)                                   # the exchange: cut globals only
            sigma[cut] = st.numpy()
            x = np.clip((sigma - M.c) / (rho * ntot), M.lb, M.ub)
            pos = 0
            xs_new = np.empty_like(xs)
            for idx, Ab, bb in blocks:
                n = len(idx)
                d = -rho * x[gk[pos:pos + n]] - lam[pos:pos + n]
                xs_new[pos:pos + n] = Ab @ d / rho + bb
                pos += n
            r = x[gk] - xs_new
            lam = lam + rho * r
            mine_g = np.unique(gk)
            sums = torch.tensor([r @ r, (xs_new - xs) @ (xs_new - xs), x[gk] @ x[gk], xs_new @ xs_new, lam @ lam,
                                 float(M.c[mine_g][owner[mine_g] == rank] @ x[mine_g][owner[mine_g] == rank])],
                                dtype=torch.float64)
            xs = xs_new
            dist.all_reduce(sums)
            iters = t + 1
            if eps_rel > 0 and iters % 50 == 0:
                conv, _ = opf.apply_test_rule(sums.numpy(), rho, eps_rel, 1e30)
                if conv:
                    break
        out[rank] = (slots, xs, lam, x, iters, conv, float(sums[5]), np.unique(gk))
    finally:
        dist.destroy_process_group()


def _run_ranks(n_iter, eps_rel):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_admm, args=(r, 2, port, out, n_iter, eps_rel)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    return dict(out)


def test_two_gloo_ranks_reproduce_the_unsharded_iterates():
    out = _run_ranks(100, 0.0)
    M = lindist.build(synth.preset_feeder("123", 2001))
    ref = oracle_admm.admm(oracle_admm.Prepared(M), rho=100.0, max_iter=100, check_every=0, record=True)
    xs = np.zeros_like(ref.xs)
    lam = np.zeros_like(ref.lam)
    for r in range(2):
        slots, xsr, lamr, x, iters, _, _, mine_g = out[r]
        xs[slots], lam[slots] = xsr, lamr
        assert np.max(np.abs(x[mine_g] - ref.x[mine_g])) <= 1e-12 * max(1.0, np.max(np.abs(ref.x)))
    assert np.max(np.abs(xs - ref.xs)) <= 1e-12 * max(1.0, np.max(np.abs(ref.xs)))
    assert np.max(np.abs(lam - ref.lam)) <= 1e-12 * max(1.0, np.max(np.abs(ref.lam)))
    assert out[0][6] == pytest.approx(ref.hist[99, 4], rel=1e-12)     # objective summed over owners


def test_two_gloo_ranks_stop_where_the_oracle_stops():
    out = _run_ranks(200_000, 1e-3)
    M = lindist.build(synth.preset_feeder("123", 2001))
    ref = oracle_admm.admm(oracle_admm.Prepared(M), rho=100.0, eps_rel=1e-3, eps_abs_pres=1e30, max_iter=200_000,
                           check_every=50)
    assert out[0][5] and out[1][5]
    assert out[0][4] == out[1][4] == ref.iters
