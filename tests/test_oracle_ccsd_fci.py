"""Pins of the CCSD / MP2 / FCI references used to judge the flow."""
import numpy as np

from oracle import ccsd, fci
from oracle.secondq import Operators, apply_string, reference_state, sector_basis
from paper_2606_04186_gb300 import synth


def test_first_iteration_is_mp2():
    eps, h, g = synth.make_system(12, 4, 3.0, 21)
    no, nv = 4, 8
    e0, r1, r2 = ccsd.residuals(h, g, np.zeros((no, nv)), np.zeros((no, no, nv, nv)), no)
    assert abs(e0 - ccsd.hf_energy(h, g, no)) < 1e-13
    assert np.abs(r1).max() < 1e-13                       # canonical RHF: no singles at first
    eo, ev = eps[:no], eps[no:]
    d2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    t2 = r2 / d2
    e1, _, _ = ccsd.residuals(h, g, np.zeros((no, nv)), t2, no)
    assert abs((e1 - e0) - ccsd.mp2_energy(eps, g, no)) < 1e-14


def test_ccsd_equals_fci_for_two_electrons():
    eps, h, g = synth.make_system(6, 1, 2.0, 4)
    g = 4.0 * g                                             # stronger correlation for a sharper test
    e_cc, *_ = ccsd.ccsd(h, g, 1, tol=1e-12)
    e_fci = fci.fci_energy(h, g, 1)
    assert abs(e_cc - e_fci) < 1e-10


def test_fci_dense_equals_lanczos():
    eps, h, g = synth.make_system(6, 3, 2.0, 8)
    a = fci.fci_energy(h, g, 3)
    b = fci.fci_energy(h, g, 3, dense_limit=0)
    assert abs(a - b) < 1e-10


def test_residuals_equal_determinant_space_similarity_transform(n10):
    # <mu| e^{-T} H e^{T} |Phi> in the 14,400-determinant space of the ten-orbital system
    eps, h, g, _ = n10
    n, no = 10, 3
    t1, t2 = synth.random_amplitudes(no, n - no, 17, 0.05, 0.05)
    ops = Operators(sector_basis(n, no, no))
    phi = reference_state(n, no)
    r = ops.apply_hbar(h, g, t1, t2, no, ops.basis.unit(phi))
    idx = ops.basis.index

    def elem(opslist):
        c, s = apply_string(opslist, phi)
        return c * r[int(idx(s))]

    e0, r1, r2 = ccsd.residuals(h, g, t1, t2, no)
    assert abs(r[int(idx(phi))] - e0) < 1e-12
    for i in range(no):
        for a in range(n - no):
            A = no + a
            assert abs(elem([("+", A), ("-", i)]) - r1[i, a]) < 1e-12
            for j in range(no):
                for b in range(n - no):
                    B = no + b
                    d = elem([("+", A), ("+", B + n), ("-", j + n), ("-", i)])
                    assert abs(d - r2[i, j, a, b]) < 1e-12
