"""Pins of the dressed Hamiltonian H-bar_<=2 (Eqs. 5-6, N = 1, SES-CC reading).

``oracle.hbar_brute`` evaluates the definition (exact e^{-T} H e^{T} in Fock space, normal
ordered, <= two-body); the closed-form spin-free ``oracle.hbar`` must agree with it on
every block.  The T = 0 and T1-only limits are further tied to textbook closed forms.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import hbar
from oracle.hbar_brute import HbarBrute
from paper_2606_04186_gb300 import synth


def _system(n, no, seed=11):
    eps, h, g = synth.make_system(n, no, 2.0, seed)
    return eps, h, g


def test_bare_limit_is_hf_fock_and_eri():
    eps, h, g = _system(4, 2)
    t1 = np.zeros((2, 2)); t2 = np.zeros((2, 2, 2, 2))
    hb = HbarBrute(h, g, t1, t2, 2)
    o = slice(0, 2)
    ehf = 2 * np.trace(h[o, o]) + 2 * np.einsum("kkll->", g[o, o, o, o]) - np.einsum("kllk->", g[o, o, o, o])
    assert abs(hb.E0 - ehf) < 1e-13
    assert np.abs(hb.spin_free_fock() - np.diag(eps)).max() < 1e-13
    assert np.abs(hb.fbar[:4, 4:]).max() == 0.0            # no spin-flip one-body part
    assert np.abs(hb.wbar() - g).max() < 1e-13


def test_t1_only_is_orbital_similarity_transform():
    # e^{-T1} H e^{T1} is exactly two-body: integrals transformed by expm(-K) / expm(K).
    n, no = 5, 2
    eps, h, g = _system(n, no)
    t1, _ = synth.random_amplitudes(no, n - no, 3, 0.1, 0.0)
    K = np.zeros((n, n)); K[no:, :no] = t1.T
    X, Y = scipy.linalg.expm(-K), scipy.linalg.expm(K)
    ht = X @ h @ Y
    gt = np.einsum("pP,Qq,rR,Ss,PQRS->pqrs", X, Y, X, Y, g)
    hb = HbarBrute(h, g, t1, np.zeros((no, no, n - no, n - no)), no)
    assert np.abs(hb.wbar() - gt).max() < 1e-13
    o = slice(0, no)
    f = ht + 2 * np.einsum("pqkk->pq", gt[:, :, o, o]) - np.einsum("pkkq->pq", gt[:, o, o, :])
    assert np.abs(hb.spin_free_fock() - f).max() < 1e-13


@pytest.mark.parametrize("n,no,mode", [(4, 2, "both"), (5, 2, "t2"), (5, 2, "both"), (6, 3, "both")])
def test_closed_form_matches_definition(n, no, mode):
    eps, h, g = _system(n, no)
    t1, t2 = synth.random_amplitudes(no, n - no, 5, 0.05, 0.05)
    if mode == "t2":
        t1 = 0 * t1
    hb = HbarBrute(h, g, t1, t2, no)
    e0, F, W = hbar.hbar2(h, g, t1, t2, no)
    assert abs(hb.E0 - e0) < 1e-12
    assert np.abs(hb.spin_free_fock() - F).max() < 1e-12
    assert np.abs(hb.wbar() - W).max() < 1e-12


def test_pair_symmetry():
    eps, h, g = _system(7, 3)
    t1, t2 = synth.random_amplitudes(3, 4, 9, 0.05, 0.05)
    _, _, W = hbar.hbar2(h, g, t1, t2, 3)
    assert np.abs(W - W.transpose(2, 3, 0, 1)).max() < 1e-14
