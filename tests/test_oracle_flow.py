"""Pins of the flow: ordering, ownership, sweep fixed point, convergence to CCSD."""
import json
import os

import numpy as np
import pytest

from oracle import ccsd, flow
from paper_2606_04186_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")


def test_paper_counts():
    gold = json.load(open(GOLDEN))
    assert flow.qubits(3, 3) == gold["active_space_33_qubits"]["value"]
    pr = gold["propane_ccpvdz"]["value"]
    assert flow.qubits(pr["No"], pr["Nv"]) == pr["qubits"]
    assert round(flow.spin_orbital_parameters(pr["No"], pr["Nv"]) / 1e6, 2) == pr["parameters"] / 1e6
    assert flow.qubits(0, gold["h2o_ccpvqz_orbitals"]["value"]) == gold["h2o_table1_qubits"]["value"]["cc-pVQZ"]


@pytest.mark.parametrize("name", ["n10", "n24"])
def test_owners_unique_and_covering(name):
    eps, h, g, sp = synth.system_inputs(name)
    s = synth.SYSTEMS[name]
    no, nv = s.nocc, s.n - s.nocc
    f = flow.Flow.__new__(flow.Flow)
    perm = flow.sort_spaces(sp, ccsd.fock_diagonal(h, g, no))
    own1, own2 = flow.owner_maps(sp[perm], no, nv)
    assert (own1 >= 0).all() and (own2 >= 0).all()
    assert np.array_equal(own2, own2.transpose(1, 0, 3, 2))
    # number of distinct amplitudes owned, summed over spaces, equals the unique count
    pairs = {(min((i, a), (j, b)), max((i, a), (j, b))) for i in range(no) for j in range(no)
             for a in range(nv) for b in range(nv)}
    assert own1.size + len(pairs) == flow.spatial_parameters(no, nv)
    # owner is the first space (in sorted order) that reaches the amplitude: brute force
    ssp = sp[perm]
    for (i, a), (j, b) in list(pairs)[:300]:
        first = next(k for k, r in enumerate(ssp)
                     if {i, j} <= set(r[2:5]) and {a + no, b + no} <= set(r[5:8]))
        assert own2[i, j, a, b] == first


def test_sort_is_input_order_independent(n10):
    eps, h, g, sp = n10
    fd = ccsd.fock_diagonal(h, g, 3)
    p1 = flow.sort_spaces(sp, fd)
    rng = np.random.default_rng(1)
    q = rng.permutation(len(sp))
    p2 = flow.sort_spaces(sp[q], fd)
    assert np.array_equal(sp[p1], sp[q][p2])
    de = [flow.delta_eps(r, fd) for r in sp[p1]]
    assert all(x <= y for x, y in zip(de, de[1:]))


def test_ccsd_amplitudes_are_a_fixed_point(n10):
    eps, h, g, sp = n10
    e_cc, t1, t2, _ = ccsd.ccsd(h, g, 3, tol=1e-13)
    f = flow.Flow(h, g, 3, sp, t1=t1, t2=t2)
    e, de, dt, nf = f.sweep()
    assert nf == 0 and dt < 1e-10
    assert np.abs(f.energies - e_cc).max() < 1e-10


def test_first_sweep_sees_bare_hamiltonian_and_energies_differ(n10):
    eps, h, g, sp = n10
    f = flow.Flow(h, g, 3, sp)
    f.sweep()
    ehf = ccsd.hf_energy(h, g, 3)
    assert np.all(f.energies < ehf)                    # each CASCI lies below HF
    assert np.ptp(f.energies) > 1e-6                   # E(i) differ between spaces


@pytest.mark.parametrize("use_diis", [False, True])
def test_flow_converges_to_ccsd(n10, use_diis):
    eps, h, g, sp = n10
    e_cc, t1, t2, _ = ccsd.ccsd(h, g, 3, tol=1e-13)
    f = flow.Flow(h, g, 3, sp, diis=use_diis)
    hist = f.run(tol_e=1e-10, tol_t=1e-9, max_sweeps=40)
    assert abs(hist[-1][1]) < 1e-10
    assert abs(f.e_mean - e_cc) < 1e-9
    assert np.abs(f.t2 - t2).max() < 1e-8 and np.abs(f.t1 - t1).max() < 1e-8
    # the paper's convergence picture: per-space changes shrink sweep over sweep
    des = [abs(x[1]) for x in hist[1:]]
    assert des[-1] < des[0]


# ---- wave-ordered sweeps (the progressive pool update of the Numerical Implementation) --------

def test_waves_wider_than_the_list_are_the_jacobi_sweep(n10):
    eps, h, g, sp = n10
    fj = flow.Flow(h, g, 3, sp)
    fw = flow.Flow(h, g, 3, sp)
    for _ in range(2):
        rj = fj.sweep()
        rw = fw.sweep_waves(len(sp))
        assert rj[0] == rw[0] and rj[2] == rw[2]
        assert np.array_equal(fj.energies, fw.energies)
        assert np.array_equal(fj.t1, fw.t1) and np.array_equal(fj.t2, fw.t2)


@pytest.mark.parametrize("wave", [1, 4])
def test_waves_keep_the_ccsd_fixed_point(n10, wave):
    eps, h, g, sp = n10
    e_cc, t1, t2, _ = ccsd.ccsd(h, g, 3, tol=1e-13)
    f = flow.Flow(h, g, 3, sp, t1=t1, t2=t2)
    e, de, dt, nf = f.sweep_waves(wave)
    assert nf == 0 and dt < 1e-10
    assert np.abs(f.energies - e_cc).max() < 1e-10


def test_first_wave_sees_the_bare_hamiltonian_and_the_second_the_first_ones_pool(n10):
    """Wave 1 (spaces 0..K-1) solves on the bare Hamiltonian like a Jacobi first sweep; wave 2
    solves on the pool those K spaces leave, which a Jacobi sweep over just those K spaces
    (they own the same amplitudes: owners are taken in list order) reproduces."""
    eps, h, g, sp = n10
    K = 5
    fw = flow.Flow(h, g, 3, sp)
    fw.sweep_waves(K)
    fj = flow.Flow(h, g, 3, sp)
    fj.sweep()
    assert np.array_equal(fw.energies[:K], fj.energies[:K])
    first = flow.Flow(h, g, 3, fw.spaces[:K])   # already sorted: keeps the order and the owners
    first.sweep()
    e0, F, W = first.dress()
    for s in range(K, 2 * K):
        occ, vir = flow.space_orbitals(fw.spaces[s])
        e_ref = flow.cas.solve_space(e0, F, W, occ, vir)[0]
        assert abs(fw.energies[s] - e_ref) < 1e-12
    assert np.abs(fw.energies[K:2 * K] - fj.energies[K:2 * K]).max() > 1e-6


@pytest.fixture(scope="module")
def jacobi_run(n10):
    eps, h, g, sp = n10
    f = flow.Flow(h, g, 3, sp)
    return f.run(tol_e=1e-10, tol_t=1e-9, max_sweeps=40)


def test_waves_converge_to_ccsd(n10, jacobi_run):
    eps, h, g, sp = n10
    e_cc, t1, t2, _ = ccsd.ccsd(h, g, 3, tol=1e-13)
    f = flow.Flow(h, g, 3, sp)
    hist = []
    for _ in range(40):
        e, de, dt, nf = f.sweep_waves(5)
        hist.append((e, de, dt))
        if abs(de) < 1e-10 and dt < 1e-9:
            break
    assert abs(f.e_mean - e_cc) < 1e-9
    assert np.abs(f.t2 - t2).max() < 1e-8 and np.abs(f.t1 - t1).max() < 1e-8
    assert len(hist) <= len(jacobi_run)   # the progressive update needs no more sweeps than Jacobi
