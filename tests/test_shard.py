"""Sharded sweeps on the CPU: the library's host shard planner against an independent
reconstruction of the partition, and a two-rank gloo run of the sharded sweep protocol with the
oracle doing each rank's per-space work.

The protocol under test: every rank dresses the same pool, solves the spaces of its shard,
writes the exchange vector [owned pool entries | energy | code] (code = status * 2^20 + Davidson
iterations, an exact integer in FP64) with -0.0 in every
entry it did not produce, the ranks sum the vectors (allreduce), and every rank merges the sum.
Owners are unique (Numerical Implementation: each amplitude belongs to exactly one space), so the
result must equal an unsharded sweep bit for bit.
"""
import math
import multiprocessing as mp
import socket

import numpy as np
import pytest

from oracle import ccsd, flow
from paper_2606_04186_gb300 import synth


@pytest.fixture(scope="module")
def qf():
    from paper_2606_04186_gb300 import build, qflow
    import os
    if not os.path.exists(qflow.LIB_PATH):
        build.build()
    qflow.lib()
    return qflow


def reference_partition(h, g, nocc, sp, rank, nranks):
    """Space and pool masks of shard `rank`, rebuilt here from the definition: device order =
    size class, then (occupied tuple, virtual tuple, sorted position); rank r takes positions
    [floor(r c / R), floor((r + 1) c / R)) of each class."""
    n = h.shape[0]
    nv = n - nocc
    perm = flow.sort_spaces(sp, ccsd.fock_diagonal(h, g, nocc))
    srt = sp[perm]
    smask = np.zeros(len(sp), dtype=np.uint8)
    for k in (1, 2, 3):
        pos = [s for s in range(len(srt)) if srt[s, 0] == k]
        pos.sort(key=lambda s: (tuple(int(x) for x in srt[s, 2:2 + 2 * k]), s))
        c = len(pos)
        for s in pos[c * rank // nranks:c * (rank + 1) // nranks]:
            smask[s] = 1
    o1, o2 = flow.owner_maps(srt, nocc, nv)
    own = np.concatenate([o1.ravel(), o2.ravel()])
    pmask = np.where(own >= 0, smask[np.maximum(own, 0)], 0).astype(np.uint8)
    return smask, pmask


@pytest.mark.parametrize("name,per_class", [("n10", 20), ("n24", 300)])
def test_shard_plan_partition(qf, name, per_class):
    s = synth.SYSTEMS[name]
    _, h, g, _ = synth.system_inputs(name, with_spaces=False)
    sp = synth.mixed_spaces(s.n, s.nocc, per_class, seed=7)
    perm, o1, o2, _ = qf.plan(h, g, s.nocc, sp)
    owned = np.concatenate([o1.ravel(), o2.ravel()]) >= 0
    for R in (1, 2, 3, 5):
        ssum = np.zeros(len(sp), dtype=np.int64)
        psum = np.zeros(owned.size, dtype=np.int64)
        for r in range(R):
            sm, pm = qf.shard_plan(h, g, s.nocc, sp, r, R)
            rs, rp = reference_partition(h, g, s.nocc, sp, r, R)
            assert np.array_equal(sm, rs) and np.array_equal(pm, rp), (R, r)
            # equal shares of every size class (within one space)
            for k in (1, 2, 3):
                cls = sp[perm][:, 0] == k
                c = int(cls.sum())
                assert int(sm[cls].sum()) in (c // R, c // R + 1)
            ssum += sm
            psum += pm
        assert np.all(ssum == 1)
        assert np.array_equal(psum, owned.astype(np.int64))


def test_shard_plan_rejects_bad_rank(qf):
    _, h, g, sp = synth.system_inputs("n10")
    for r, R in ((0, 0), (2, 2), (-1, 3)):
        with pytest.raises(qf.QFlowError):
            qf.shard_plan(h, g, 3, sp, r, R)


# ---- two ranks over gloo ----------------------------------------------------------------------

def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pack(t1n, t2n, res, smask, pmask):
    """Exchange vector of one rank; -0.0 where the rank produced nothing."""
    ns = len(res)
    pool = np.concatenate([t1n.ravel(), t2n.ravel()])
    x = np.full(pool.size + 2 * ns, -0.0)
    x[:pool.size] = np.where(pmask == 1, pool, -0.0)
    e = np.array([r[0] if r is not None else 0.0 for r in res])
    st = np.array([float(int(r[3]) << 20) if r is not None else 0.0 for r in res])
    x[pool.size:pool.size + ns] = np.where(smask == 1, e, -0.0)
    x[pool.size + ns:pool.size + 2 * ns] = np.where(smask == 1, st, -0.0)
    return x


def _rank_main(rank, nranks, port, sweeps, q):
    import torch
    import torch.distributed as dist
    from paper_2606_04186_gb300 import qflow
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=nranks)
    try:
        s = synth.SYSTEMS["n10"]
        _, h, g, _ = synth.system_inputs("n10", with_spaces=False)
        sp = synth.mixed_spaces(s.n, s.nocc, 12, seed=7)
        smask, pmask = qflow.shard_plan(h, g, s.nocc, sp, rank, nranks)
        fl = flow.Flow(h, g, s.nocc, sp)
        t1, t2 = fl.t1, fl.t2
        out = []
        for _ in range(sweeps):
            e0, F, W = hbar_dress(h, g, t1, t2, s.nocc)
            res = [flow.cas.solve_space(e0, F, W, *flow.space_orbitals(row)) if smask[i] else None
                   for i, row in enumerate(fl.spaces)]
            # spaces of other shards contribute nothing (their increments are masked out)
            filled = [r if r is not None else (0.0, np.zeros((k, k)), np.zeros((k, k, k, k)), 0)
                      for r, k in zip(res, fl.spaces[:, 0])]
            t1n, t2n = flow.merge(t1, t2, fl.spaces, filled, fl.own1, fl.own2, s.nocc)
            x = torch.from_numpy(_pack(t1n, t2n, res, smask, pmask))
            dist.all_reduce(x, op=dist.ReduceOp.SUM)
            x = x.numpy()
            npool = t1.size + t2.size
            own = np.concatenate([fl.own1.ravel(), fl.own2.ravel()])
            pool_old = np.concatenate([t1.ravel(), t2.ravel()])
            pool = np.where(own >= 0, x[:npool], pool_old)
            t1 = pool[:t1.size].reshape(t1.shape)
            t2 = pool[t1.size:].reshape(t2.shape)
            energies = x[npool:npool + len(sp)]
            out.append((pool.copy(), energies.copy(), float(np.mean(energies))))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def hbar_dress(h, g, t1, t2, nocc):
    from oracle import hbar
    return hbar.hbar2(h, g, t1, t2, nocc)


def test_two_rank_gloo_sweeps_equal_unsharded():
    """World size 2 over gloo: two sharded sweeps equal the oracle's unsharded sweeps bitwise."""
    pytest.importorskip("torch")
    from paper_2606_04186_gb300 import build, qflow
    import os
    if not os.path.exists(qflow.LIB_PATH):
        build.build()
    sweeps = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, sweeps, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = synth.SYSTEMS["n10"]
    _, h, g, _ = synth.system_inputs("n10", with_spaces=False)
    sp = synth.mixed_spaces(s.n, s.nocc, 12, seed=7)
    ref = flow.Flow(h, g, s.nocc, sp)
    for k in range(sweeps):
        e_mean, _, _, _ = ref.sweep()
        pool_ref = np.concatenate([ref.t1.ravel(), ref.t2.ravel()])
        for r in (0, 1):
            pool, energies, em = got[r][k]
            assert np.array_equal(pool, pool_ref), (r, k)
            assert np.array_equal(energies, ref.energies), (r, k)
            assert em == e_mean
    # the shards really split the work
    m0, _ = qflow.shard_plan(h, g, s.nocc, sp, 0, 2)
    assert 0 < int(m0.sum()) < len(sp)
    assert math.isfinite(e_mean)
