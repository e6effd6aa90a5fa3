"""Sharded sweeps on one GPU: R handles, each solving its shard, their exchange vectors summed on
the device (what an allreduce over R processes computes), must reproduce the unsharded sweep bit
for bit: energies, pool, convergence scalars and per-space statistics, sweep after sweep.
Owners are unique (Numerical Implementation), so every exchanged entry has exactly one producer."""
import numpy as np
import pytest

from paper_2606_04186_gb300 import synth

from gpu_util import library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


def _sharded_sweep(flows, bufs):
    import torch
    for f, x in zip(flows, bufs):
        f.sweep_shard_begin(x)
    total = bufs[0].clone()
    for x in bufs[1:]:
        total += x
    for x in bufs:
        x.copy_(total)
    torch.cuda.synchronize()
    return [f.sweep_shard_end(x) for f, x in zip(flows, bufs)]


@pytest.mark.parametrize("name,precision,R,diis,guess", [
    ("n24", "fp64", 2, 0, "phi"),
    ("n40", "fp64", 3, 0, "phi"),
    ("n40", "mixed", 3, 6, "previous"),
    ("n40", "mixed", 2, 0, "phi"),
    ("n40", "mixed", 1, 0, "phi"),
])
def test_sharded_sweeps_bitwise(qf, name, precision, R, diis, guess):
    import torch
    s = synth.SYSTEMS[name]
    _, h, g, sp = synth.system_inputs(name)
    ref = qf.Flow(h, g, s.nocc, sp, precision=precision, diis=diis, guess=guess)
    flows = [qf.Flow(h, g, s.nocc, sp, precision=precision, diis=diis, guess=guess) for _ in range(R)]
    for r, f in enumerate(flows):
        f.set_shard(r, R)
    n = flows[0].exchange_size()
    assert n == s.nocc * (s.n - s.nocc) + (s.nocc * (s.n - s.nocc)) ** 2 + 2 * len(sp)
    bufs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(R)]
    for sweep in range(3):
        de, dt, nf, code = ref.sweep()
        outs = _sharded_sweep(flows, bufs)
        e_ref, per_ref = ref.energy(per_space=True)
        t1r, t2r = ref.amplitudes()
        it_ref, st_ref = ref.stats()
        for r, (f, out) in enumerate(zip(flows, outs)):
            assert out[2] == nf and out[3] == code, (sweep, r)
            assert out[1] == dt, (sweep, r)
            if sweep > 0:
                assert out[0] == de, (sweep, r)
            e, per = f.energy(per_space=True)
            assert e == e_ref and np.array_equal(per, per_ref), (sweep, r)
            t1, t2 = f.amplitudes()
            assert np.array_equal(t1, t1r) and np.array_equal(t2, t2r), (sweep, r)
            it, st = f.stats()
            assert np.array_equal(it, it_ref) and np.array_equal(st, st_ref), (sweep, r)
    for f in flows + [ref]:
        f.close()


def test_shard_call_order(qf):
    import torch
    s = synth.SYSTEMS["n10"]
    _, h, g, sp = synth.system_inputs("n10")
    f = qf.Flow(h, g, s.nocc, sp, precision="mixed")
    x = torch.empty(f.exchange_size(), dtype=torch.float64, device="cuda")
    with pytest.raises(qf.QFlowError) as ei:  # no shard set
        f.sweep_shard_begin(x)
    assert ei.value.code == qf.ERR_STATE
    f.set_shard(0, 2)
    assert f.sweep(raise_on_fail=False)[3] == qf.ERR_STATE  # plain sweep refused when sharded
    with pytest.raises(qf.QFlowError):
        f.sweep_shard_end(x)  # end before begin
    f.sweep_shard_begin(x)
    with pytest.raises(qf.QFlowError):
        f.sweep_shard_begin(x)  # begin twice
    t1, t2 = f.amplitudes()
    with pytest.raises(qf.QFlowError):
        f.set_amplitudes(t1, t2)  # pool is being swept
    with pytest.raises(qf.QFlowError):
        f.set_shard(1, 2)
    f.sweep_shard_end(x, raise_on_fail=False)
    with pytest.raises(qf.QFlowError):
        f.set_shard(2, 2)
    f.set_shard(0, 1)  # back to the whole list, still through begin / end
    f.sweep_shard_begin(x)
    f.sweep_shard_end(x)
    f.close()
