"""Parity at the benchmark sizes (n82: all 7,156,800 (3,3) spaces; n114: 2,000,000 sampled spaces)
in the launch configuration the benchmark uses, on sampled outputs the oracle computes one by
one: the first sweep starts from the empty pool, where the dressed Hamiltonian is the bare one
(E0 = E_HF, F = the Fock matrix, W = the integrals), so each sampled space's energy and
increment are a CASCI solve of the oracle on the bare integrals."""
import numpy as np
import pytest

from oracle import cas, ccsd, flow
from paper_2606_04186_gb300 import synth

from gpu_util import library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


@pytest.mark.parametrize("name", ["n82", "n114"])
def test_first_sweep_sampled_spaces_match_oracle(qf, name):
    s = synth.SYSTEMS[name]
    _, h, g, sp = synth.system_inputs(name)
    no, nv = s.nocc, s.n - s.nocc
    fl = qf.Flow(h, g, no, sp, precision="mixed")
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
    rng = np.random.default_rng(0)
    for pos in rng.choice(len(sp), 24, replace=False):
        occ, vir = flow.space_orbitals(sp[perm[pos]])
        e_ref, x1, x2, st = cas.solve_space(e_hf, F, g, occ, vir)
        assert st == 0
        assert abs(per[pos] - e_ref) < 1e-6, (pos, per[pos], e_ref)
        va = [a - no for a in vir]
        for ii, i in enumerate(occ):        # increments of the amplitudes this space owns
            for aa, a in enumerate(va):
                if o1[i, a] == pos:
                    assert abs(t1[i, a] - x1[ii, aa]) < 1e-5
            for jj, j in enumerate(occ):
                for aa, a in enumerate(va):
                    for bb, b in enumerate(va):
                        if o2[i, j, a, b] == pos:
                            assert abs(t2[i, j, a, b] - x2[ii, jj, aa, bb]) < 1e-5
