"""GPU parity of the sharded single instance (opf_shard_*) through the C ABI.

Several shards of one feeder run on one GPU as the ranks of a multi-GPU
solve would (one shard per rank): every iteration each shard enqueues its
part of the cut globals' sigma, the parts are added (the all-reduce of a
multi-GPU run, here a device sum after all shards finished their part: no
kernel waits on another), and each shard runs its iteration with the sums.

* x, x_s and lambda after 100 FP64 iterations equal the unsharded oracle's
  within 1e-10 relative, for 2 to 4 shards of the 13-, 123- and 8500-bus
  feeders;
* the Sec. III-C sums added over the shards give the oracle's residuals and
  objective, and the shards stop at the oracle's iteration.
"""
import numpy as np
import pytest

from oracle import admm as oracle_admm, lindist
from paper_2310_09410_gb300 import opf, synth

pytestmark = pytest.mark.gpu

RHO = 100.0


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run_shards(f, n_parts, n_iter, check_every=50, eps_rel=0.0):
    import torch
    M = lindist.build(f)
    part = opf.partition(f, n_parts, len(M.subs))
    shards = [opf.Shard(f, part, p) for p in range(n_parts)]
    try:
        for sh in shards:
            sh.precompute()
        C = shards[0].n_cut
        for sh in shards:
            assert sh.n_cut == C and np.array_equal(sh.cut_global, shards[0].cut_global)
        dev = torch.device("cuda", 0)
        sig = [torch.zeros(max(C, 1), dtype=torch.float64, device=dev) for _ in shards]
        sums = [torch.zeros(6, dtype=torch.float64, device=dev) for _ in shards]
        tot = torch.zeros(max(C, 1), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        it, conv, out = 0, False, None
        while it < n_iter:
            for sh, sg in zip(shards, sig):
                sh.partial(RHO, sg.data_ptr())
            torch.cuda.synchronize()
            tot.copy_(torch.stack(sig).sum(0))               # the exchange over the cut
            torch.cuda.synchronize()
            it += 1
            check = check_every > 0 and it % check_every == 0
            for sh, sm in zip(shards, sums):
                sh.step(RHO, tot.data_ptr(), sm.data_ptr() if check else None)
            torch.cuda.synchronize()
            if check:
                total = torch.stack(sums).sum(0).cpu().numpy()
                conv, out = opf.apply_test_rule(total, RHO, eps_rel if eps_rel > 0 else 1.0, 1e30)
                if eps_rel > 0 and conv:
                    break
        res = [(sh.global_of_local.copy(), sh.x(), *sh.locals()) for sh in shards]
    finally:
        for sh in shards:
            sh.close()
    return M, part, res, it, conv, out


def assemble(M, part, res):
    """x_s, lambda in the oracle's slot order (subsystems in canonical order;
    a shard lists its subsystems' slots in the same order)."""
    P = oracle_admm.Prepared(M)
    xs = np.full(int(P.off[-1]), np.nan)
    lam = np.full_like(xs, np.nan)
    for p, (_, _, xsp, lamp) in enumerate(res):
        pos = 0
        for s in range(len(M.subs)):
            if part[s] != p:
                continue
            n = int(P.off[s + 1] - P.off[s])
            xs[P.off[s]:P.off[s + 1]] = xsp[pos:pos + n]
            lam[P.off[s]:P.off[s + 1]] = lamp[pos:pos + n]
            pos += n
        assert pos == len(xsp)
    return xs, lam


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


@pytest.mark.parametrize("name,seed,n_parts", [("13", 1001, 2), ("123", 2001, 2), ("123", 2001, 4),
                                               ("8500", 3001, 4)])
def test_shards_match_oracle_iterates(name, seed, n_parts):
    f = synth.preset_feeder(name, seed)
    M, part, res, it, _, out = run_shards(f, n_parts, 100)
    ref = oracle_admm.admm(oracle_admm.Prepared(M), rho=RHO, max_iter=100, check_every=0, record=True)
    xs, lam = assemble(M, part, res)
    assert rel(xs, ref.xs) <= 1e-10
    assert rel(lam, ref.lam) <= 1e-10
    for gl, x, _, _ in res:
        assert rel(x, ref.x[gl]) <= 1e-10
    want = ref.hist[99]
    for k in range(5):
        assert abs(out[k] - want[k]) <= 1e-10 * max(abs(want[k]), 1e-300), (k, out[k], want[k])


@pytest.mark.parametrize("name,seed,n_parts", [("13", 1001, 2), ("123", 2001, 3)])
def test_shards_stop_where_the_oracle_stops(name, seed, n_parts):
    f = synth.preset_feeder(name, seed)
    M, part, res, it, conv, _ = run_shards(f, n_parts, 200_000, check_every=50, eps_rel=1e-3)
    ref = oracle_admm.admm(oracle_admm.Prepared(M), rho=RHO, eps_rel=1e-3, eps_abs_pres=1e30, max_iter=200_000,
                           check_every=50)
    assert conv and ref.converged
    assert it == ref.iters


def test_shard_errors():
    f = synth.preset_feeder("13", 1001)
    M = lindist.build(f)
    part = opf.partition(f, 2, len(M.subs))
    with pytest.raises(opf.OPFError):
        opf.Shard(f, part, 5)                    # no such part
    with opf.Shard(f, part, 0) as sh:
        with pytest.raises(opf.OPFError) as e:
            sh.step(RHO, None)                   # before precompute / partial
        assert e.value.code in (opf.OPF_E_STATE, opf.OPF_E_INVALID)
