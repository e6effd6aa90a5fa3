"""Pins of the DUCC-form oracle (oracle/ducc.py): the truncated commutator, the operators it is
applied to, the per-space decomposition, and the flow built on it."""
import numpy as np
import pytest

from oracle import cas, ducc, flow, hbar
from oracle.secondq import apply_string
from paper_2606_04186_gb300 import synth


# ---- brute force on the Fock space of a few spin orbitals ---------------------------------------

def _fock_matrix(ops, nso: int, phi: int):
    """Matrix of the normal-ordered (with respect to phi) string `ops` on all 2^nso states."""
    qc, qa = [], []
    for pos, (kind, P) in enumerate(ops):
        filled = (phi >> P) & 1
        creates = (kind == "+" and not filled) or (kind == "-" and filled)
        (qc if creates else qa).append(pos)
    order = qc + qa
    inv = sum(1 for i in range(len(order)) for j in range(i + 1, len(order)) if order[i] > order[j])
    sign = -1.0 if inv & 1 else 1.0
    nops = [ops[k] for k in order]
    dim = 1 << nso
    mat = np.zeros((dim, dim))
    for s in range(dim):
        c, t = apply_string(nops, s)
        if c:
            mat[t, s] += sign * c
    return mat


def _operator_matrix(op, nso: int, phi: int):
    c, f, v = op
    dim = 1 << nso
    mat = c * np.eye(dim)
    for P in range(nso):
        for Q in range(nso):
            if f[P, Q]:
                mat += f[P, Q] * _fock_matrix([("+", P), ("-", Q)], nso, phi)
    for P in range(nso):
        for Q in range(nso):
            for R in range(nso):
                for S in range(nso):
                    if v[P, Q, R, S]:
                        mat += 0.25 * v[P, Q, R, S] * _fock_matrix([("+", P), ("+", Q), ("-", S), ("-", R)], nso, phi)
    return mat


def _random_operator(rng, nso):
    f = rng.standard_normal((nso, nso))
    v = rng.standard_normal((nso,) * 4)
    v = v - v.transpose(1, 0, 2, 3)
    v = v - v.transpose(0, 1, 3, 2)
    return float(rng.standard_normal()), f, v


@pytest.mark.parametrize("phi", [0b000111, 0b001011, 0b000000, 0b110101])
def test_commutator_matches_exact_commutator_below_three_body(phi):
    # Wick's theorem: the exact [A, B] of two two-body operators is its normal-ordered 0..3-body
    # parts; a three-body part moves six quasi-particles, so it cannot connect states whose
    # quasi-particle counts (bits flipped from phi) add up to five or less.  On all those elements
    # the truncated commutator must equal the exact one.
    nso = 6
    rng = np.random.default_rng(phi)
    A, B = _random_operator(rng, nso), _random_operator(rng, nso)
    occ = np.array([(phi >> P) & 1 for P in range(nso)], dtype=float)
    C = ducc.commutator(A, B, occ)
    ma, mb = _operator_matrix(A, nso, phi), _operator_matrix(B, nso, phi)
    exact = ma @ mb - mb @ ma
    got = _operator_matrix(C, nso, phi)
    dim = 1 << nso
    qp = np.array([bin(s ^ phi).count("1") for s in range(dim)])
    mask = (qp[:, None] + qp[None, :]) <= 5
    assert np.abs(exact - got)[mask].max() < 1e-11
    assert np.abs(exact - got).max() > 1e-3   # the dropped three-body part is really there


# ---- the operators and the per-space decomposition ------------------------------------------------

def test_h_t_commutator_is_the_t_linear_part_of_the_ses_cc_dressing(n10):
    # e^{-T} H e^{T} = H + [H, T] + 1/2 [[H, T], T] + ... is a polynomial of degree 4 in T, so its
    # T-linear part is the five-point central difference in lambda of the SES-CC dressing of
    # lambda T (exact for degree 4); the <=2-body truncation is linear, so it must equal
    # [H, T]_(<=2) from the commutator formula.
    eps, h, g, _ = n10
    no, n = 3, 10
    t1, t2 = synth.random_amplitudes(no, n - no, 21, 0.05, 0.08)
    d = {lam: hbar.hbar2(h, g, lam * t1, lam * t2, no) for lam in (-2.0, -1.0, 1.0, 2.0)}
    lin = [(8.0 * (d[1.0][k] - d[-1.0][k]) - (d[2.0][k] - d[-2.0][k])) / 12.0 for k in range(3)]
    H = ducc.hamiltonian(h, g, no)
    tf, tv = ducc.cluster(t1, t2, no, n)
    e0, F, W = ducc.spin_free(ducc.commutator(H, (0.0, tf, tv), ducc.occupations(n, no)), n)
    assert abs(e0 - lin[0]) < 1e-11
    assert np.abs(F - lin[1]).max() < 1e-11
    assert np.abs(W - lin[2]).max() < 1e-11


def test_hamiltonian_and_sigma_in_spin_orbitals(n10):
    # H normal ordered: E_HF and the Fock matrix; the spin-free two-body part is (pq|rs).  sigma is
    # anti-Hermitian and its excitation part is T.
    eps, h, g, _ = n10
    no, n = 3, 10
    c, f, v = ducc.hamiltonian(h, g, no)
    e0, F, W = ducc.spin_free((c, f, v), n)
    assert abs(e0 - hf_energy(h, g, no)) < 1e-13
    assert np.abs(F - np.diag(eps)).max() < 1e-12
    assert np.abs(W - g).max() < 1e-15
    t1, t2 = synth.random_amplitudes(no, n - no, 4)
    _, sf, sv = ducc.sigma_operator(t1, t2, no, n)
    assert np.abs(sf + sf.T).max() == 0.0 and np.abs(sv + sv.transpose(2, 3, 0, 1)).max() == 0.0
    # <Phi_ij^ab (alpha beta)| T |Phi>: W-convention element v[a_alpha, b_beta, i_alpha, j_beta] = t2[i, j, a, b]
    assert np.abs(sv[no:n, n + no:, :no, n:n + no] - t2.transpose(2, 3, 0, 1)).max() == 0.0


def hf_energy(h, g, no):
    from oracle import ccsd
    return ccsd.hf_energy(h, g, no)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_decomposition_equals_the_definition(n10, k):
    # G|_A - L_A must equal the truncated transform computed from sigma_ext directly.
    eps, h, g, _ = n10
    no, n = 3, 10
    t1, t2 = synth.random_amplitudes(no, n - no, 8, 0.04, 0.06)
    d = ducc.Dressing(h, g, t1, t2, no)
    sp = synth.all_spaces(n, no, k, k)
    for row in sp[:: max(1, len(sp) // 6)]:
        occ, vir = flow.space_orbitals(row)
        a = d.space_operator(occ, vir)
        b = d.space_operator_direct(occ, vir)
        assert abs(a[0] - b[0]) < 1e-12
        assert np.abs(a[1] - b[1]).max() < 1e-12 and np.abs(a[2] - b[2]).max() < 1e-12
        # Hermitian, and sigma_int really changes it (the internal part is not in sigma_ext)
        assert np.abs(a[1] - a[1].T).max() < 1e-12
        assert np.abs(a[2] - a[2].transpose(2, 3, 0, 1)).max() < 1e-12
        idx = ducc.active_spin_orbitals(list(occ) + list(vir), n)
        gA = ducc.restrict(d.G, idx)
        assert np.abs(gA[2] - a[2]).max() > 1e-6


def test_first_sweep_is_the_ses_cc_first_sweep(n10):
    # empty pool: sigma = 0, H_eff = the bare Hamiltonian of each space (CASCI), and the new
    # internal amplitudes equal the SES-CC increments from zero
    eps, h, g, sp = n10
    a = ducc.Flow(h, g, 3, sp)
    b = flow.Flow(h, g, 3, sp)
    ea, *_ = a.sweep()
    eb, *_ = b.sweep()
    assert abs(ea - eb) < 1e-12
    assert np.abs(a.energies - b.energies).max() < 1e-11
    assert np.abs(a.t1 - b.t1).max() < 1e-11 and np.abs(a.t2 - b.t2).max() < 1e-11


def test_full_space_gives_fci_every_sweep():
    # one space holding every orbital: sigma_ext = 0 at every sweep, so H_eff = H and E = FCI
    from oracle import fci
    eps, h, g = synth.make_system(4, 2, 2.0, 31)
    g = 3.0 * g
    sp = synth.all_spaces(4, 2, 2, 2)
    assert len(sp) == 1
    e_fci = fci.fci_energy(h, g, 2)
    fl = ducc.Flow(h, g, 2, sp)
    for _ in range(3):
        e, de, dt, nf = fl.sweep()
        assert nf == 0 and abs(e - e_fci) < 1e-11


def test_truncation_is_exact_through_second_order_without_interaction():
    # H = F (one-body, diagonal): e^{-S} F e^{S} = F + [F, S] + 1/2 [[F, S], S] + O(S^3), so on the
    # elements no three-body term reaches the truncated transform differs from the exact one by
    # O(lambda^3) for S -> lambda S; with an interaction the difference is O(lambda^2) (the
    # fluctuation potential's double commutator is left out).
    from scipy.linalg import expm
    nso, phi = 6, 0b000111
    rng = np.random.default_rng(3)
    occ = np.array([(phi >> P) & 1 for P in range(nso)], dtype=float)
    fd = np.diag(np.sort(rng.standard_normal(nso)))
    A = _random_operator(rng, nso)
    S = (0.0, A[1] - A[1].T, A[2] - A[2].transpose(2, 3, 0, 1))
    dim = 1 << nso
    qp = np.array([bin(s ^ phi).count("1") for s in range(dim)])
    mask = (qp[:, None] + qp[None, :]) <= 5
    V = _random_operator(rng, nso)
    V = (0.0, 0.0 * V[1], 0.5 * (V[2] + V[2].transpose(2, 3, 0, 1)))
    for with_v, order in ((False, 3), (True, 2)):
        H = (0.0, fd, V[2] if with_v else np.zeros((nso,) * 4))
        mh, ms = _operator_matrix(H, nso, phi), _operator_matrix(S, nso, phi)
        errs = []
        for lam in (0.02, 0.01):
            exact = expm(-lam * ms) @ mh @ expm(lam * ms)
            trunc = _operator_matrix(ducc.truncated_transform(H, ducc.scale(S, lam), occ), nso, phi)
            errs.append(np.abs(exact - trunc)[mask].max())
        assert 0.8 * 2 ** order < errs[0] / errs[1] < 1.25 * 2 ** order, errs


def test_flow_energies_hermitian_and_converging(n10):
    eps, h, g, sp = n10
    fl = ducc.Flow(h, g, 3, sp)
    hist = [fl.sweep() for _ in range(8)]
    assert all(hh[3] == 0 for hh in hist)
    de = [abs(hh[1]) for hh in hist[1:]]
    assert de[-1] < 1e-6 and de[-1] < de[0]
    d = ducc.Dressing(h, g, fl.t1, fl.t2, 3)
    occ, vir = flow.space_orbitals(fl.spaces[0])
    _, _, _, _, asym = ducc.solve_space(d.space_operator(occ, vir), 3, 3)
    assert asym < 1e-12
