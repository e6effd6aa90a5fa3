"""The Hermitian (DUCC) form on the GPU against the oracle (oracle/ducc.py), through the C ABI.

* The SES-CC dressing kernels applied to B = [F, sigma] (an operator without the integrals'
  (pq|rs) = (qp|rs) symmetry) equal the oracle's dressing of it: the DUCC form builds its common
  part from the T-linear parts of such dressings.
* DUCC flows (FP64) match the oracle's sweep by sweep: 10 orbitals, every (3,3) space and a list
  mixing the three size classes; 24 orbitals (every (3,3) space on the GPU, a seeded sample of
  spaces recomputed by the oracle) from a seeded pool.
Tolerances: FP64, 1e-9 Eh and 1e-9 on amplitudes (1e-8 at 24 orbitals).
"""
import numpy as np
import pytest

from oracle import ducc, flow, hbar
from paper_2606_04186_gb300 import synth

from gpu_util import dev, library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


@pytest.mark.parametrize("name", ["n10", "n24"])
def test_dressing_kernels_on_the_sigma_commutator(qf, name):
    import torch
    eps, h, g, _ = synth.system_inputs(name, with_spaces=False)
    s = synth.SYSTEMS[name]
    n, no = s.n, s.nocc
    t1, t2 = synth.random_amplitudes(no, n - no, 17, 0.03, 0.05)
    occ = ducc.occupations(n, no)
    H = ducc.hamiltonian(h, g, no)
    B = ducc.commutator(ducc.fock_part(H), ducc.sigma_operator(t1, t2, no, n), occ)
    _, hb, gb = ducc.spin_free(B, n)
    e0r, Fr, Wr = hbar.hbar2(hb, gb, t1, t2, no)
    e0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    W = torch.zeros((n,) * 4, dtype=torch.float64, device="cuda")
    work = torch.zeros(qf.dress_workspace(n, no), dtype=torch.uint8, device="cuda")
    qf.dress_device(dev(hb), dev(gb), dev(t1), dev(t2), no, e0, F, W, work)
    torch.cuda.synchronize()
    assert abs(e0.item() - e0r) < 1e-11
    assert np.abs(F.cpu().numpy() - Fr).max() < 1e-11
    assert np.abs(W.cpu().numpy() - Wr).max() < 1e-11


def _mixed_list(n, no):
    return np.concatenate([synth.all_spaces(n, no, k, k) for k in (3, 2, 1)])


@pytest.mark.parametrize("spaces", ["all33", "mixed"])
def test_ducc_flow_matches_oracle(qf, spaces):
    eps, h, g, sp = synth.system_inputs("n10")
    if spaces == "mixed":
        sp = _mixed_list(10, 3)
    ref = ducc.Flow(h, g, 3, sp)
    gpu = qf.Flow(h, g, 3, sp, precision="fp64", form="ducc")
    assert np.array_equal(gpu.order(), ref.perm)
    for sweep in range(4):
        er, der, dtr, nfr = ref.sweep()
        de, dt, nf, code = gpu.sweep()
        e, per = gpu.energy(per_space=True)
        t1, t2 = gpu.amplitudes()
        assert nf == nfr == 0 and code == 0
        assert abs(e - er) < 1e-9
        assert np.abs(per - ref.energies).max() < 1e-9
        assert np.abs(t1 - ref.t1).max() < 1e-9 and np.abs(t2 - ref.t2).max() < 1e-9
    gpu.close()


def test_ducc_first_sweep_is_the_ses_cc_first_sweep(qf):
    eps, h, g, sp = synth.system_inputs("n24")
    a = qf.Flow(h, g, 5, sp, precision="fp64", form="ducc")
    b = qf.Flow(h, g, 5, sp, precision="fp64")
    a.sweep()
    b.sweep()
    ea, pa = a.energy(per_space=True)
    eb, pb = b.energy(per_space=True)
    assert np.abs(pa - pb).max() < 1e-10
    assert np.abs(a.amplitudes()[1] - b.amplitudes()[1]).max() < 1e-10
    a.close()
    b.close()


def _mp2_pool(h, g, no, seed):
    """t2[i,j,a,b] = (ia|jb) / (e_i + e_j - e_a - e_b), e the Fock diagonal; small seeded singles."""
    from oracle import ccsd
    n = h.shape[0]
    e = ccsd.fock_diagonal(h, g, no)
    den = e[:no, None, None, None] + e[None, :no, None, None] - e[None, None, no:, None] - e[None, None, None, no:]
    t2 = np.ascontiguousarray(g[:no, no:, :no, no:].transpose(0, 2, 1, 3) / den)
    return synth.random_amplitudes(no, n - no, seed, scale1=0.005)[0], t2


def test_ducc_sweep_n24_sampled_spaces(qf):
    eps, h, g, sp = synth.system_inputs("n24")
    no, nv = 5, 19
    t1, t2 = _mp2_pool(h, g, no, 3)
    gpu = qf.Flow(h, g, no, sp, precision="fp64", form="ducc")
    gpu.set_amplitudes(t1, t2)
    de, dt, nf, code = gpu.sweep(raise_on_fail=False)
    e, per = gpu.energy(per_space=True)
    it, st_gpu = gpu.stats()
    t1n, t2n = gpu.amplitudes()
    perm = gpu.order()
    sps = sp[perm]
    own1, own2 = flow.owner_maps(sps, no, nv)
    d = ducc.Dressing(h, g, t1, t2, no)
    rng = np.random.default_rng(5)
    n_owned = 0
    for s_idx in rng.choice(len(sps), size=40, replace=False):
        occ, vir = flow.space_orbitals(sps[s_idx])
        er, x1, x2, st, asym = ducc.solve_space(d.space_operator(occ, vir), 3, 3)
        assert asym < 1e-12
        assert (st_gpu[s_idx] != 0) == (st != 0), (s_idx, st_gpu[s_idx], st)
        if st != 0:
            continue
        assert abs(per[s_idx] - er) < 1e-8
        va = [a - no for a in vir]
        for ii, i in enumerate(occ):
            for aa, a in enumerate(va):
                if own1[i, a] == s_idx:
                    n_owned += 1
                    assert abs(t1n[i, a] - x1[ii, aa]) < 1e-8
            for jj, j in enumerate(occ):
                for aa, a in enumerate(va):
                    for bb, b in enumerate(va):
                        if own2[i, j, a, b] == s_idx:
                            n_owned += 1
                            assert abs(t2n[i, j, a, b] - x2[ii, jj, aa, bb]) < 1e-8
    assert n_owned > 0
    assert nf == int((st_gpu != 0).sum()) and nf <= len(sp) // 1000
    gpu.close()


def test_ducc_form_arguments(qf):
    eps, h, g, sp = synth.system_inputs("n10")
    with pytest.raises(qf.QFlowError):
        qf.Flow(h, g, 3, sp, precision="mixed", form="ducc")
    fl = qf.Flow(h, g, 3, sp, precision="fp64", form="ducc")
    with pytest.raises(qf.QFlowError) as err:
        fl.sweep_waves(5)
    assert err.value.code == qf.ERR_STATE
    fl.close()
