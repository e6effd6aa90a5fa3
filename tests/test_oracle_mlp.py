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


def test_adam_first_step_is_the_normalised_gradient():
    # Kingma and Ba (2015), Algorithm 1: at t = 1 the bias-corrected moments are m = g and v = g*g,
    # so every parameter moves by -lr * g / (|g| + eps), whatever beta1 and beta2 are.
    rng = np.random.default_rng(5)
    p = rng.standard_normal(40)
    g = rng.standard_normal(40) * np.logspace(-3, 2, 40)
    z = np.zeros(40)
    p1, m1, v1 = mlp.adam_step(p, g, z, z, 1, 0.05)
    np.testing.assert_allclose(p1 - p, -0.05 * g / (np.abs(g) + 1e-8), rtol=1e-13, atol=0.0)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)  # 1 - 0.9 rounds
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_adam_second_step_hand_computed():
    # One scalar parameter, p0 = 0.5, gradients g1 = 1 then g2 = -2, lr = 0.1, betas (0.9, 0.999),
    # eps = 1e-8, worked by hand from Kingma and Ba (2015), Algorithm 1:
    #   t = 1: m = 0.1, v = 0.001, m^ = 1, v^ = 1               -> p1 = 0.5 - 0.1 / (1 + 1e-8)
    #   t = 2: m = 0.09 - 0.2 = -0.11, v = 0.000999 + 0.004 = 0.004999,
    #          m^ = -0.11 / 0.19 = -11/19, v^ = 0.004999 / 0.001999 = 4999/1999
    #                                                           -> p2 = p1 + 0.1 (11/19) / (sqrt(4999/1999) + 1e-8)
    # Swapping the betas or dropping either bias correction changes p2 in the third digit.
    p = np.array([0.5])
    z = np.zeros(1)
    p1, m, v = mlp.adam_step(p, np.array([1.0]), z, z, 1, 0.1)
    p2, m, v = mlp.adam_step(p1, np.array([-2.0]), m, v, 2, 0.1)
    want1 = 0.5 - 0.1 / (1.0 + 1e-8)
    want2 = want1 + 0.1 * (11.0 / 19.0) / (np.sqrt(4999.0 / 1999.0) + 1e-8)
    assert abs(p1[0] - want1) < 1e-15
    assert abs(m[0] - (-0.11)) < 1e-15 and abs(v[0] - 0.004999) < 1e-17
    assert abs(p2[0] - want2) < 1e-14
    assert abs(want2 - 0.4366103534720748) < 1e-15
