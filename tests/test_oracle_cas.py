"""Pins of the per-space problem: downfolded operator, root, CI -> CC increment."""
import numpy as np
import scipy.linalg

from oracle import cas, fci, hbar
from oracle.secondq import Operators, cas_operators, reference_state, sector_basis
from paper_2606_04186_gb300 import synth


def _bare(h, g, nocc):
    return hbar.hbar2(h, g, np.zeros((nocc, h.shape[0] - nocc)),
                      np.zeros((nocc, nocc, h.shape[0] - nocc, h.shape[0] - nocc)), nocc)


def test_full_space_is_fci():
    for n, no in [(4, 2), (6, 3)]:
        eps, h, g = synth.make_system(n, no, 2.0, 31)
        e0, F, W = _bare(h, g, no)
        e, x1, x2, st = cas.solve_space(e0, F, W, list(range(no)), list(range(no, n)))
        assert st == 0
        assert abs(e - fci.fci_energy(h, g, no)) < 1e-10


def test_bare_space_is_frozen_core_casci():
    # T = 0: the space operator equals the projection of the full Hamiltonian onto the
    # determinants with inactive orbitals doubly occupied and external virtuals empty.
    n, no = 8, 4
    eps, h, g = synth.make_system(n, no, 2.0, 5)
    occ, vir = [1, 2, 3], [4, 6, 7]
    e0, F, W = _bare(h, g, no)
    c, hh, w = cas.space_problem(e0, F, W, occ, vir)
    mat = cas.cas_matrix(3, 3, c, hh, w)
    full = Operators(sector_basis(n, no, no))
    cops = cas_operators(3, 3)
    act = occ + vir
    core = [0]
    cols = []
    for s in cops.basis.states:
        a, b = int(s) & 63, int(s) >> 6
        fa = sum(1 << act[k] for k in range(6) if a >> k & 1) | sum(1 << k for k in core)
        fb = sum(1 << act[k] for k in range(6) if b >> k & 1) | sum(1 << k for k in core)
        cols.append(int(full.basis.index(fa | (fb << n))))
    proj = np.empty((400, 400))
    eye = np.eye(full.basis.dim)
    for k, col in enumerate(cols):
        proj[:, k] = full.apply_hamiltonian(0.0, h, g, eye[:, col])[cols]
    # same operator up to a +-1 diagonal basis phase: equal |elements| and equal spectra
    assert np.abs(np.abs(mat) - np.abs(proj)).max() < 1e-12
    assert np.abs(np.sort(np.linalg.eigvalsh(mat)) - np.sort(np.linalg.eigvalsh(proj))).max() < 1e-11


def test_root_matches_scipy_eig_and_is_phi_dominant():
    n, no = 9, 4
    eps, h, g = synth.make_system(n, no, 3.0, 6)
    t1, t2 = synth.random_amplitudes(no, n - no, 2, 0.03, 0.03)
    e0, F, W = hbar.hbar2(h, g, t1, t2, no)
    c, hh, w = cas.space_problem(e0, F, W, [0, 2, 3], [4, 5, 8])
    mat = cas.cas_matrix(3, 3, c, hh, w)
    _, _, _, phi = cas.coupling(3, 3)
    e, vec, st = cas.phi_root(mat, phi)
    assert st == 0 and vec[phi] == 1.0
    assert np.linalg.norm(mat @ vec - e * vec) < 1e-10 * np.linalg.norm(vec)
    ws, vs = scipy.linalg.eig(mat)
    k = np.argmax(np.abs(vs[phi]))
    assert abs(ws[k].real - e) < 1e-10 and abs(ws[k].imag) < 1e-12
    assert abs(e - min(np.real(ws))) < 1e-10  # weakly correlated: the Phi-dominant root is the lowest


def test_ci_to_cc_round_trip():
    # c = e^{T_int} Phi built exactly in the space; the increment read from it returns T_int.
    for no, nv in [(1, 1), (2, 2), (3, 3)]:
        ops = cas_operators(no, nv)
        t1, t2 = synth.random_amplitudes(no, nv, 40 + no, 0.2, 0.2)
        phi = reference_state(no + nv, no)
        vec = ops.apply_exp_cluster(t1, t2, no, ops.basis.unit(phi), +1.0)
        x1, x2 = cas.increment(no, nv, vec)
        assert np.abs(x1 - t1).max() < 1e-13
        assert np.abs(x2 - t2).max() < 1e-13
