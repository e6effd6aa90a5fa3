"""Hermitian (DUCC) form of the downfolded Hamiltonian and the flow built on it.  Test
infrastructure only: nothing in the product path imports or runs this module.

The paper's downfolding uses an anti-Hermitian sigma (Eq. 1) and, with N = 1 in Eqs. 5-8, the
effective Hamiltonian of active space A_i is the projection of e^{-sigma_ext} H e^{sigma_ext} onto
the space's determinants (its internal part sigma_int is what the active-space solver determines).
The paper computes it with DUCC and states neither the commutator truncation nor the many-body
truncation, so this module fixes them (a reading):

    H_eff(i) = P_i [ H + [H, s] + 1/2 [[F, s], s] ]_(<=2) P_i,   s = sigma_ext(i) = T_ext - T_ext^+,

* T is the closed-shell singles-and-doubles pool, T_ext(i) its amplitudes with at least one index
  outside A_i;
* F is the Fock operator of the reference, diagonal in the canonical orbitals: counting F as zeroth
  order and the fluctuation potential and s as first order, these are all terms through second
  order (the double commutator of the fluctuation potential is third order and left out);
* [.]_(<=2): every commutator is normal ordered with respect to Phi and kept to its zero-, one- and
  two-body parts (its three-body part dropped);
* the space's root is the eigenvector with the largest |c_Phi| (the operator is Hermitian);
* the internal amplitudes are read from that root through the cluster map C1 = t1,
  C2 = t2 + t1^2 / 2 (the paper's VQE returns UCCSD parameters directly; the cluster amplitudes of
  the root equal them to first order), and they replace the owned pool amplitudes.

Decomposition used to evaluate it (exact within the truncation): with sigma = T - T^+ the whole
pool and sigma_int(i) its internal part,
    H_eff(i) = G|_A - L_A,   G = [H + [H, sigma] + 1/2 [[F, sigma], sigma]]_(<=2),
    L_A = [H_A + ... : [H_A, sigma_int] + 1/2 [[F_A, sigma_int], sigma_int]]_(<=2),
where X|_A keeps the terms of X whose indices all lie in A and H_A, F_A are H, F restricted to A:
in a commutator with an operator whose indices are all in A, contractions run over indices of A
and the other factor's free indices are output indices, so only its restriction to A enters; F is
diagonal, so [F, sigma]|_A = [F, sigma_int].  G is computed once per sweep, L_A per space on the
space's 12 spin orbitals.  Both routes are compared in the tests.

Representation: spin orbitals alpha 0..n-1, beta n..2n-1; a normal-ordered operator is
(c, f[P,Q], v[P,Q,R,S]) for c + sum f_PQ {P+ Q} + 1/4 sum v_PQRS {P+ Q+ S R}, v antisymmetric in
(P, Q) and in (R, S).  Spin-free results: F_pq = f[p_alpha, q_alpha] and
W_pqrs = v[p_alpha, r_beta, q_alpha, s_beta] (creators p, r; annihilators q, s), as oracle.hbar.

Parity pins (tests/test_oracle_ducc.py): the commutator equals the exact Fock-space commutator on
every matrix element a three-body operator cannot reach; [H, T] equals the T-linear part of the
SES-CC dressing (oracle.hbar); the two routes to H_eff agree; sigma = 0 gives the bare
Hamiltonian (first sweep = the SES-CC first sweep = CASCI); H_eff is Hermitian; a space that holds
every orbital gives FCI at every sweep; with no two-body interaction the truncation is the exact
similarity transformation through second order.
"""
from __future__ import annotations

import numpy as np

from .cas import cas_matrix, coupling, increment, unnormal_order
from .flow import owner_maps, sort_spaces, space_orbitals
from .ccsd import fock_diagonal, hf_energy


# ---- spin-orbital operators --------------------------------------------------------------------

def occupations(n: int, nocc: int) -> np.ndarray:
    occ = np.zeros(2 * n)
    occ[:nocc] = 1.0
    occ[n:n + nocc] = 1.0
    return occ


def _antisym(x: np.ndarray) -> np.ndarray:
    """(1 - P_PQ)(1 - P_RS) x for x[P,Q,R,S]."""
    return x - x.transpose(1, 0, 2, 3) - x.transpose(0, 1, 3, 2) + x.transpose(1, 0, 3, 2)


def hamiltonian(h: np.ndarray, g: np.ndarray, nocc: int):
    """H = c + sum h E + 1/2 sum (pq|rs)(E E - delta E), normal ordered with respect to Phi."""
    n = h.shape[0]
    m = 2 * n
    fs = h + 2.0 * np.einsum("pqkk->pq", g[:, :, :nocc, :nocc]) - np.einsum("pkkq->pq", g[:, :nocc, :nocc, :])
    f = np.zeros((m, m))
    f[:n, :n] = fs
    f[n:, n:] = fs
    # <PR|QS> = (pq|rs) delta(spin P, spin Q) delta(spin R, spin S), stored as d[P,R,Q,S]
    d = np.zeros((m, m, m, m))
    gt = g.transpose(0, 2, 1, 3)   # [p, r, q, s]
    for sp in (0, n):
        for sr in (0, n):
            d[sp:sp + n, sr:sr + n, sp:sp + n, sr:sr + n] = gt
    v = d - d.transpose(0, 1, 3, 2)
    return hf_energy(h, g, nocc), f, v


def cluster(t1: np.ndarray, t2: np.ndarray, nocc: int, n: int):
    """T = sum t_i^a E_ai + 1/2 sum t_ij^ab E_ai E_bj as (f, v) with v[A,B,I,J] = <AB||IJ> amplitudes."""
    m = 2 * n
    f = np.zeros((m, m))
    v = np.zeros((m, m, m, m))
    occ = [np.arange(nocc), np.arange(nocc) + n]
    vir = [np.arange(nocc, n), np.arange(nocc, n) + n]
    for s in (0, 1):
        f[np.ix_(vir[s], occ[s])] = t1.T
    ab = t2.transpose(2, 3, 0, 1)   # [a, b, i, j]
    for s1 in (0, 1):
        for s2 in (0, 1):
            blk = np.zeros((m, m, m, m))
            blk[np.ix_(vir[s1], vir[s2], occ[s1], occ[s2])] = ab
            v += blk - blk.transpose(0, 1, 3, 2)
    return f, v


def sigma_operator(t1, t2, nocc: int, n: int):
    """sigma = T - T^+ (anti-Hermitian)."""
    f, v = cluster(t1, t2, nocc, n)
    return 0.0, f - f.T, v - v.transpose(2, 3, 0, 1)


def commutator(A, B, occ: np.ndarray):
    """[A, B] normal ordered with respect to the reference with occupations `occ`, truncated to its
    zero-, one- and two-body parts (Wick's theorem; the three-body part is dropped)."""
    _, a1, a2 = A
    _, b1, b2 = B
    n_ = occ
    nb = 1.0 - occ
    # zero-body
    c0 = float(np.einsum("pq,qp,pq->", a1, b1, n_[:, None] - n_[None, :]))
    hhpp = np.einsum("p,q,r,s->pqrs", n_, n_, nb, nb)
    c0 += 0.25 * float(np.sum((a2 * b2.transpose(2, 3, 0, 1) - b2 * a2.transpose(2, 3, 0, 1)) * hhpp))
    # one-body
    c1 = a1 @ b1 - b1 @ a1
    dn = n_[:, None] - n_[None, :]   # n_r - n_s
    c1 += np.einsum("rs,sprq->pq", a1 * dn, b2) - np.einsum("rs,sprq->pq", b1 * dn, a2)
    w3 = (np.einsum("r,s,t->rst", n_, n_, nb) + np.einsum("r,s,t->rst", nb, nb, n_))
    c1 += 0.5 * (np.einsum("tprs,rstq,rst->pq", a2, b2, w3, optimize=True)
                 - np.einsum("tprs,rstq,rst->pq", b2, a2, w3, optimize=True))
    # two-body
    x = np.einsum("pt,tqrs->pqrs", a1, b2) - np.einsum("pt,tqrs->pqrs", b1, a2)
    c2 = x - x.transpose(1, 0, 2, 3)
    y = np.einsum("tr,pqts->pqrs", a1, b2) - np.einsum("tr,pqts->pqrs", b1, a2)
    c2 -= y - y.transpose(0, 1, 3, 2)
    w2 = 1.0 - n_[:, None] - n_[None, :]
    c2 += 0.5 * (np.einsum("pqtu,tu,turs->pqrs", a2, w2, b2, optimize=True)
                 - np.einsum("pqtu,tu,turs->pqrs", b2, w2, a2, optimize=True))
    z = np.einsum("ab,bjal,aibk->ijkl", dn, a2, b2, optimize=True)
    c2 -= _antisym(z)
    return c0, c1, c2


def add(*terms):
    c = sum(t[0] for t in terms)
    return c, sum(t[1] for t in terms), sum(t[2] for t in terms)


def scale(A, s: float):
    return s * A[0], s * A[1], s * A[2]


def fock_part(H):
    """The diagonal of H's one-body part (the Fock operator in canonical orbitals)."""
    m = H[1].shape[0]
    return 0.0, np.diag(np.diag(H[1])), np.zeros((m,) * 4)


def truncated_transform(H, S, occ):
    """[H + [H, S] + 1/2 [[F, S], S]]_(<=2) with F the diagonal of H's one-body part."""
    F = fock_part(H)
    return add(H, commutator(H, S, occ), scale(commutator(commutator(F, S, occ), S, occ), 0.5))


def spin_free(op, n: int):
    """(E0, F, W) of a spin-free operator in spin-orbital form."""
    c, f, v = op
    return c, f[:n, :n].copy(), v[:n, n:, :n, n:].transpose(0, 2, 1, 3).copy()


# ---- the per-space operator ----------------------------------------------------------------------

def active_spin_orbitals(orbs, n: int) -> np.ndarray:
    orbs = list(orbs)
    return np.array(orbs + [p + n for p in orbs])


def restrict(op, idx: np.ndarray):
    c, f, v = op
    return c, f[np.ix_(idx, idx)], v[np.ix_(idx, idx, idx, idx)]


def embed_internal(S, idx: np.ndarray):
    """The part of S whose indices all lie in idx (as a full-size operator)."""
    c, f, v = S
    fi = np.zeros_like(f)
    vi = np.zeros_like(v)
    fi[np.ix_(idx, idx)] = f[np.ix_(idx, idx)]
    vi[np.ix_(idx, idx, idx, idx)] = v[np.ix_(idx, idx, idx, idx)]
    return 0.0, fi, vi


class Dressing:
    """H, sigma and the global part G of one sweep (spin-orbital)."""

    def __init__(self, h, g, t1, t2, nocc: int):
        self.n = n = h.shape[0]
        self.nocc = nocc
        self.occ = occupations(n, nocc)
        self.H = hamiltonian(h, g, nocc)
        self.S = sigma_operator(t1, t2, nocc, n)
        self.G = truncated_transform(self.H, self.S, self.occ)

    def space_operator(self, occ_orbs, vir_orbs):
        """Spin-orbital H_eff of a space on its own spin orbitals: G|_A - L_A."""
        idx = active_spin_orbitals(list(occ_orbs) + list(vir_orbs), self.n)
        HA = restrict(self.H, idx)
        SA = restrict(self.S, idx)
        L = truncated_transform(HA, SA, self.occ[idx])
        L = (L[0] - HA[0], L[1] - HA[1], L[2] - HA[2])   # the commutator terms only
        GA = restrict(self.G, idx)
        return GA[0] - L[0], GA[1] - L[1], GA[2] - L[2]

    def space_operator_direct(self, occ_orbs, vir_orbs):
        """The same operator from its definition: the truncated transform with sigma_ext."""
        idx = active_spin_orbitals(list(occ_orbs) + list(vir_orbs), self.n)
        Sint = embed_internal(self.S, idx)
        Sext = (0.0, self.S[1] - Sint[1], self.S[2] - Sint[2])
        return restrict(truncated_transform(self.H, Sext, self.occ), idx)


def space_problem(op_active, no: int):
    """(c, h, w) of the space's CAS operator from its spin-orbital operator on 2 (no + nv) spin
    orbitals (local order: occupied then virtual, alpha then beta)."""
    m = op_active[1].shape[0] // 2
    e0, F, W = spin_free(op_active, m)
    c, h = unnormal_order(e0, F, W, no)
    return c, h, W


def solve_space(op_active, no: int, nv: int):
    """Energy, internal amplitudes (X1, X2) and status of one space: the root with the largest
    |c_Phi| of the (symmetric) CAS matrix, normalised to c_Phi = 1, through the cluster map."""
    c, h, w = space_problem(op_active, no)
    mat = cas_matrix(no, nv, c, h, w)
    _, _, _, phi = coupling(no, nv)
    sym = 0.5 * (mat + mat.T)
    ev, vec = np.linalg.eigh(sym)
    k = int(np.argmax(np.abs(vec[phi, :])))
    x = vec[:, k]
    status = 0 if abs(x[phi]) >= 1e-3 else 1
    x1, x2 = increment(no, nv, x / x[phi])
    return float(ev[k]), x1, x2, status, float(np.abs(mat - mat.T).max())


class Flow:
    """QFlow in the DUCC reading: Jacobi sweeps from an empty pool; the owners' internal
    amplitudes replace the pool's (unowned amplitudes and flagged spaces leave them unchanged)."""

    def __init__(self, h, g, nocc: int, spaces, t1=None, t2=None):
        self.h, self.g, self.nocc = h, g, nocc
        n = h.shape[0]
        self.nvir = n - nocc
        self.perm = sort_spaces(spaces, fock_diagonal(h, g, nocc))
        self.spaces = np.asarray(spaces)[self.perm]
        self.own1, self.own2 = owner_maps(self.spaces, nocc, self.nvir)
        self.t1 = np.zeros((nocc, self.nvir)) if t1 is None else t1.copy()
        self.t2 = np.zeros((nocc, nocc, self.nvir, self.nvir)) if t2 is None else t2.copy()
        self.e_mean = None
        self.energies = None

    def sweep(self):
        """One barrier-to-barrier sweep; returns (E_mean, dE, max|dt|, n_failed)."""
        d = Dressing(self.h, self.g, self.t1, self.t2, self.nocc)
        t1n, t2n = self.t1.copy(), self.t2.copy()
        energies = np.zeros(len(self.spaces))
        nfail = 0
        for s, row in enumerate(self.spaces):
            occ, vir = space_orbitals(row)
            e, x1, x2, st, _ = solve_space(d.space_operator(occ, vir), len(occ), len(vir))
            energies[s] = e
            if st != 0:
                nfail += 1
                continue
            va = [a - self.nocc for a in vir]
            for ii, i in enumerate(occ):
                for aa, a in enumerate(va):
                    if self.own1[i, a] == s:
                        t1n[i, a] = x1[ii, aa]
                for jj, j in enumerate(occ):
                    for aa, a in enumerate(va):
                        for bb, b in enumerate(va):
                            if self.own2[i, j, a, b] == s:
                                t2n[i, j, a, b] = x2[ii, jj, aa, bb]
        dt = max(np.abs(t1n - self.t1).max(initial=0.0), np.abs(t2n - self.t2).max(initial=0.0))
        self.t1, self.t2 = t1n, t2n
        self.energies = energies
        e_mean = float(np.mean(energies))
        de = float("inf") if self.e_mean is None else e_mean - self.e_mean
        self.e_mean = e_mean
        return e_mean, de, float(dt), nfail
