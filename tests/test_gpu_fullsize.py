"""Parity at the benchmark sizes (n82: all 7,156,800 (3,3) spaces; n114: 2,000,000 sampled spaces)
in the launch configuration the benchmark uses, on sampled outputs the oracle computes one by
one, in the mixed form and in the plain FP64 form.  The first sweep starts from the empty pool, where the dressed Hamiltonian is the bare one
(E0 = E_HF, F = the Fock matrix, W = the integrals), so each sampled space's energy and
increment are a CASCI solve of the oracle on the bare integrals.  A dressed sweep starts from a
pool set by the caller (MP2 doubles, the textbook first-order amplitudes, and small seeded
singles): the oracle dresses the Hamiltonian with that pool in FP64 and solves the sampled
spaces on it.  The mixed dressing itself is compared with the oracle's FP64 dressing element by
element at n82 (every E0, F and W entry: full-size tiles, grouped jobs and pipeline wrap-around of
the tensor-core engine)."""
import numpy as np
import pytest

from oracle import cas, ccsd, flow
from paper_2606_04186_gb300 import synth

from gpu_util import mixed_flow_w, library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


def _positions(o1, o2, nspaces, seed):
    """12 random sorted positions and 12 positions that own amplitudes (the owners of 4 random
    singles and 8 random doubles that have one), so that increments are checked too."""
    rng = np.random.default_rng(seed)
    pos = list(rng.choice(nspaces, 12, replace=False))
    own1 = o1[o1 >= 0]
    own2 = o2[o2 >= 0]
    pos += list(rng.choice(own1, 4, replace=False)) + list(rng.choice(own2, 8, replace=False))
    return [int(p) for p in dict.fromkeys(pos)]


TOL = {"fp64": (1e-8, 1e-7), "mixed": (1e-6, 1e-5)}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("name", ["n82", "n114"])
def test_first_sweep_sampled_spaces_match_oracle(qf, name, precision):
    s = synth.SYSTEMS[name]
    _, h, g, sp = synth.system_inputs(name)
    no, nv = s.nocc, s.n - s.nocc
    te, tt = TOL[precision]
    fl = qf.Flow(h, g, no, sp, precision=precision)
    de, dt, nf, code = fl.sweep(raise_on_fail=False)
    assert nf == 0 and code == 0
    e_mean, per = fl.energy(per_space=True)
    assert abs(e_mean - per.mean()) < 1e-9
    perm = fl.order()
    t1, t2 = fl.amplitudes()
    fl.close()
    _, o1, o2, _ = qf.plan(h, g, no, sp)
    # bare dressing: Fock matrix, E_HF
    occ_idx = np.arange(no)
    F = h + 2.0 * np.einsum("pqkk->pq", g[:, :, occ_idx][:, :, :, occ_idx]) \
        - np.einsum("pkkq->pq", g[:, occ_idx][:, :, occ_idx])
    e_hf = ccsd.hf_energy(h, g, no)
    n_owned = 0
    for pos in _positions(o1, o2, len(sp), 0):
        occ, vir = flow.space_orbitals(sp[perm[pos]])
        e_ref, x1, x2, st = cas.solve_space(e_hf, F, g, occ, vir)
        assert st == 0
        assert abs(per[pos] - e_ref) < te, (pos, per[pos], e_ref)
        va = [a - no for a in vir]
        for ii, i in enumerate(occ):        # increments of the amplitudes this space owns
            for aa, a in enumerate(va):
                if o1[i, a] == pos:
                    n_owned += 1
                    assert abs(t1[i, a] - x1[ii, aa]) < tt
            for jj, j in enumerate(occ):
                for aa, a in enumerate(va):
                    for bb, b in enumerate(va):
                        if o2[i, j, a, b] == pos:
                            n_owned += 1
                            assert abs(t2[i, j, a, b] - x2[ii, jj, aa, bb]) < tt
    assert n_owned >= 8


def _mp2_pool(h, g, no, seed):
    """t2[i,j,a,b] = (ia|jb) / (e_i + e_j - e_a - e_b) with e the Fock diagonal; t1 seeded, small."""
    n = h.shape[0]
    eps = ccsd.fock_diagonal(h, g, no)
    ovov = g[:no, no:, :no, no:]
    den = (eps[:no, None, None, None] + eps[None, :no, None, None]
           - eps[None, None, no:, None] - eps[None, None, None, no:])
    t2 = np.ascontiguousarray(ovov.transpose(0, 2, 1, 3) / den)
    t1 = synth.random_amplitudes(no, n - no, seed, scale1=0.005)[0]
    return t1, t2


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("name", ["n82", "n114"])
def test_dressed_sweep_sampled_spaces_match_oracle(qf, name, precision):
    from oracle import hbar
    s = synth.SYSTEMS[name]
    _, h, g, sp = synth.system_inputs(name)
    no = s.nocc
    te, tt = TOL[precision]
    t1_0, t2_0 = _mp2_pool(h, g, no, 3)
    fl = qf.Flow(h, g, no, sp, precision=precision)
    fl.set_amplitudes(t1_0, t2_0)
    de, dt, nf, code = fl.sweep(raise_on_fail=False)
    assert nf == 0 and code == 0
    _, per = fl.energy(per_space=True)
    perm = fl.order()
    t1, t2 = fl.amplitudes()
    fl.close()
    _, o1, o2, _ = qf.plan(h, g, no, sp)
    e0, F, W = hbar.hbar2(h, g, t1_0, t2_0, no)
    n_owned = 0
    for pos in _positions(o1, o2, len(sp), 1):
        occ, vir = flow.space_orbitals(sp[perm[pos]])
        e_ref, x1, x2, st = cas.solve_space(e0, F, W, occ, vir)
        assert st == 0
        assert abs(per[pos] - e_ref) < te, (pos, per[pos], e_ref)
        va = [a - no for a in vir]
        for ii, i in enumerate(occ):
            for aa, a in enumerate(va):
                if o1[i, a] == pos:
                    n_owned += 1
                    assert abs((t1[i, a] - t1_0[i, a]) - x1[ii, aa]) < tt
            for jj, j in enumerate(occ):
                for aa, a in enumerate(va):
                    for bb, b in enumerate(va):
                        if o2[i, j, a, b] == pos:
                            n_owned += 1
                            assert abs((t2[i, j, a, b] - t2_0[i, j, a, b]) - x2[ii, jj, aa, bb]) < tt
    assert n_owned >= 8
    # amplitudes no space owns keep the caller's values
    free2 = o2 < 0
    assert np.array_equal(t2[free2], t2_0[free2])


def test_mixed_dressing_elementwise_n82(qf):
    """Every element of the mixed dressing at n82 (E0, F, W: 45 M entries) against the oracle's
    FP64 dressing for the same pool; bounds as at n24 (E0 and F 1e-9, W 1e-6)."""
    from oracle import hbar
    s = synth.SYSTEMS["n82"]
    _, h, g, sp = synth.system_inputs("n82")
    no = s.nocc
    t1_0, t2_0 = _mp2_pool(h, g, no, 3)
    fl = qf.Flow(h, g, no, sp[:4096], precision="mixed")  # the dressing does not depend on the list
    fl.set_amplitudes(t1_0, t2_0)
    e0, F, W = fl.dressed()
    fl.close()
    e0r, Fr, Wr = hbar.hbar2(h, g, t1_0, t2_0, no)
    assert abs(e0 - e0r) < 1e-9
    assert np.abs(F - Fr).max() < 1e-9
    o, v = slice(0, no), slice(no, s.n)
    # the flow's mixed dressing adds the vvvv block's T2 term where at most three of the four
    # virtual indices differ (what (k, k) spaces with k <= 3 read)
    W = mixed_flow_w(W, Wr, no)
    for name, blk in [("oooo", (o, o, o, o)), ("vvvv", (v, v, v, v)), ("vovo", (v, o, v, o)), ("ovov", (o, v, o, v)),
                      ("vvoo", (v, v, o, o)), ("vvvo", (v, v, v, o)), ("vovv", (v, o, v, v)), ("ooov", (o, o, o, v)),
                      ("vooo", (v, o, o, o)), ("voov", (v, o, o, v))]:
        err = np.abs(W[blk] - Wr[blk]).max()
        assert err < 1e-6, (name, err)
    assert np.abs(W - Wr).max() < 1e-6
