"""Pins of the CCSD / MP2 / FCI references used to judge the flow."""
import numpy as np
import pytest

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


def _linear_map(d, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    A *= 0.9 / np.abs(np.linalg.eigvals(A)).max()  # a contraction, spectral radius 0.9
    b = rng.standard_normal(d)
    return A, b, np.linalg.solve(np.eye(d) - A, b)


@pytest.mark.parametrize("d", [1, 3, 6])
def test_diis_solves_a_linear_fixed_point_from_d_plus_one_iterates(d):
    # Pulay's extrapolation on x <- A x + b: d + 1 error vectors e_k = x_{k+1} - x_k in R^d have an
    # affine combination (coefficients summing to one) equal to zero; with those coefficients the
    # combined iterate is the fixed point (I - A)^-1 b exactly, so the push that completes d + 1
    # iterates returns it to round-off.
    from oracle.ccsd import Diis
    A, b, xstar = _linear_map(d, 10 + d)
    acc = Diis(size=8)
    x = np.random.default_rng(d).standard_normal(d)
    for k in range(d + 1):
        xn = A @ x + b
        out = acc.push(xn, xn - x)
        x = xn
    assert np.abs(out - xstar).max() < 1e-9 * max(1.0, np.abs(xstar).max())
    assert np.abs(x - xstar).max() > 1e-3  # the plain iterate is still far from it


def test_diis_history_keeps_the_newest_vectors():
    # With a history of size 3 in dimension 2, three unrelated (vector, error) pairs pushed first
    # must be gone once three iterates of the linear map follow; keeping an old pair instead of
    # a new one, or never dropping, leaves the extrapolate off the fixed point.
    from oracle.ccsd import Diis
    A, b, xstar = _linear_map(2, 7)
    rng = np.random.default_rng(8)
    acc = Diis(size=3)
    for _ in range(3):
        acc.push(rng.standard_normal(2), rng.standard_normal(2))
    x = rng.standard_normal(2)
    for _ in range(3):
        xn = A @ x + b
        out = acc.push(xn, xn - x)
        x = xn
    assert np.abs(out - xstar).max() < 1e-10


def test_diis_with_one_vector_returns_it():
    from oracle.ccsd import Diis
    acc = Diis()
    v = np.arange(4.0)
    assert acc.push(v, np.ones(4)) is v
