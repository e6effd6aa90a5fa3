"""Pins of the FP64 warm-start network reference: gradients vs central finite differences."""
import numpy as np

from oracle import mlp
from paper_2606_04186_gb300 import synth


def test_gradients_match_finite_differences():
    n_in, n_h, n_out = 7, 5, 3
    rng = np.random.default_rng(0)
    p = synth.mlp_init_params(n_in, n_h, n_out, 1) + 0.05 * rng.standard_normal(mlp.param_count(n_in, n_h, n_out))
    X = rng.standard_normal((11, n_in))
    T = rng.standard_normal((11, n_out))
    L, g = mlp.loss_and_grad(p, X, T, n_in, n_h, n_out)
    h = 1e-6
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = mlp.loss_and_grad(p + e, X, T, n_in, n_h, n_out)
        lm, _ = mlp.loss_and_grad(p - e, X, T, n_in, n_h, n_out)
        assert abs((lp - lm) / (2 * h) - g[k]) < 1e-8


def test_adam_reduces_loss():
    n_in, n_h, n_out = 6, 16, 2
    rng = np.random.default_rng(2)
    X = rng.standard_normal((64, n_in))
    T = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2]], axis=1)
    p = synth.mlp_init_params(n_in, n_h, n_out, 3)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0, _ = mlp.loss_and_grad(p, X, T, n_in, n_h, n_out)
    for t in range(1, 301):
        L, g = mlp.loss_and_grad(p, X, T, n_in, n_h, n_out)
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
    assert L < 0.2 * L0


def _space(seed=0):
    from oracle import flow, hbar
    from paper_2606_04186_gb300 import synth
    eps, h, g, sp = synth.system_inputs("n10")
    t1, t2 = synth.random_amplitudes(3, 7, seed, 0.01, 0.02)
    e0, F, W = hbar.hbar2(h, g, t1, t2, 3)
    return e0, F, W, sp


def test_guess_vector_roundtrip_rank_and_phi():
    from oracle.secondq import cas_operators, reference_state
    rng = np.random.default_rng(4)
    y = 0.1 * rng.standard_normal(mlp.N_TARGETS)
    v = mlp.guess_vector(y)
    ops = cas_operators(3, 3)
    phi = int(ops.basis.index(reference_state(6, 3)))
    assert v[phi] == 1.0
    assert np.abs(mlp.targets(v) - y).max() < 1e-14
    virt = 0b111000
    rank = np.array([bin(int(s) & virt).count("1") + bin((int(s) >> 6) & virt).count("1") for s in ops.basis.states])
    assert np.abs(v[rank > 2]).max() == 0.0
    assert np.abs(v[rank == 2]).max() > 0.0


def test_guess_vector_is_a_singlet():
    """S+ annihilates the guess: a wrong sign or a missing same-spin double would break it."""
    from oracle.secondq import Basis, excitation_matrix, sector_basis, cas_operators
    rng = np.random.default_rng(5)
    v = mlp.guess_vector(0.2 * rng.standard_normal(mlp.N_TARGETS))
    b0 = cas_operators(3, 3).basis
    big = Basis(6, list(b0.states) + list(sector_basis(6, 4, 2).states))
    w = np.zeros(big.dim)
    w[big.index(b0.states)] = v
    splus = sum(excitation_matrix(big, p, p + 6) for p in range(6))
    assert np.abs(splus @ w).max() < 1e-14
    # the check has teeth: flipping one same-spin double breaks it
    virt = 0b111000
    aa = [k for k, s in enumerate(b0.states) if bin(int(s) & virt).count("1") == 2]
    w2 = w.copy()
    w2[big.index(b0.states[aa[0]])] *= -1.0
    assert np.abs(splus @ w2).max() > 1e-6


def test_feature_packing_reproduces_cas_operator():
    from oracle import cas, flow
    e0, F, W, sp = _space()
    row = sp[sp[:, 0] == 3][5]
    occ, vir = flow.space_orbitals(row)
    x = mlp.features(e0, F, W, occ, vir)
    assert x.size == mlp.N_FEATURES
    c, h, w = cas.space_problem(e0, F, W, occ, vir)
    hf, wf, fd = mlp.unpack_features(x)
    ref = cas.cas_matrix(3, 3, c, h, w)
    mat = cas.cas_matrix(3, 3, 0.0, hf, wf)
    assert np.abs(ref - mat - c * np.eye(ref.shape[0])).max() < 1e-12
    orb = list(occ) + list(vir)
    assert np.array_equal(fd, np.diag(F)[orb])
