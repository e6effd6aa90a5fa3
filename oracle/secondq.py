"""Second quantisation on bit-string determinants (definition-level, slow, obviously correct).

Spin orbitals of an n-orbital problem are numbered alpha 0..n-1, beta n..2n-1, and a
basis state is the integer bitmask of occupied spin orbitals.  A state's sign convention
is the creation string in ascending spin-orbital order acting on the vacuum, so every
alpha creator stands left of every beta creator.  a_P and a+_P pick up (-1)^(number of
occupied spin orbitals with a lower index).

The Hamiltonian is the spin-free second-quantised operator of the paper's Eq. (1),
    H = c + sum_pq h_pq E_pq + 1/2 sum_pqrs g_pqrs (E_pq E_rs - delta_qr E_ps),
with E_pq = sum_sigma a+_{p sigma} a_{q sigma} and g_pqrs = (pq|rs).  The closed-shell
singles-and-doubles cluster operator (the SES-CC reading of sigma in Eqs. 1-8) is
    T = sum_ai t_i^a E_ai + 1/2 sum_ijab t_ij^ab E_ai E_bj.
Everything here works on explicit vectors in a determinant basis and uses nothing but
these definitions.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np
import scipy.sparse as sp


def _parity_below(states: np.ndarray, orb: int) -> np.ndarray:
    below = states & ((np.int64(1) << orb) - 1)
    return (np.bitwise_count(below) & 1).astype(np.int64)


class Basis:
    """A sorted set of bit-string states with index lookup."""

    def __init__(self, n: int, states):
        self.n = n
        self.states = np.array(sorted(set(int(s) for s in states)), dtype=np.int64)
        self.dim = self.states.size

    def index(self, s) -> np.ndarray:
        s = np.asarray(s, dtype=np.int64)
        idx = np.searchsorted(self.states, s)
        idx = np.minimum(idx, self.dim - 1)
        ok = self.states[idx] == s
        return np.where(ok, idx, -1)

    def unit(self, s: int) -> np.ndarray:
        v = np.zeros(self.dim)
        v[int(self.index(s))] = 1.0
        return v


def fock_basis(n: int) -> Basis:
    return Basis(n, range(1 << (2 * n)))


def string_masks(norb: int, nel: int):
    return [sum(1 << p for p in c) for c in itertools.combinations(range(norb), nel)]


def sector_basis(n: int, nalpha: int, nbeta: int) -> Basis:
    sa = string_masks(n, nalpha)
    sb = string_masks(n, nbeta)
    return Basis(n, [a | (b << n) for a in sa for b in sb])


def reference_state(n: int, nocc: int) -> int:
    """Closed-shell determinant with the lowest `nocc` spatial orbitals doubly occupied."""
    occ = (1 << nocc) - 1
    return occ | (occ << n)


def excitation_matrix(basis: Basis, P: int, Q: int) -> sp.csr_matrix:
    """Matrix of a+_P a_Q (spin orbitals) in `basis` (rows: result, columns: input)."""
    S = basis.states
    has_q = ((S >> Q) & 1) == 1
    cols = np.nonzero(has_q)[0]
    s0 = S[cols]
    sign = 1 - 2 * _parity_below(s0, Q)
    s1 = s0 ^ (np.int64(1) << Q)
    free_p = ((s1 >> P) & 1) == 0
    cols, s1, sign = cols[free_p], s1[free_p], sign[free_p]
    sign = sign * (1 - 2 * _parity_below(s1, P))
    s2 = s1 | (np.int64(1) << P)
    rows = basis.index(s2)
    keep = rows >= 0
    return sp.csr_matrix((sign[keep].astype(float), (rows[keep], cols[keep])), shape=(basis.dim, basis.dim))


class Operators:
    """Spin-summed unitary-group generators E_pq on a basis, and H / T applied to vectors."""

    def __init__(self, basis: Basis):
        self.basis = basis
        n = basis.n
        self.n = n
        self.E = [[excitation_matrix(basis, p, q) + excitation_matrix(basis, p + n, q + n)
                   for q in range(n)] for p in range(n)]

    def apply_one_body(self, x: np.ndarray, v: np.ndarray) -> np.ndarray:
        n = self.n
        out = np.zeros_like(v)
        for p in range(n):
            for q in range(n):
                if x[p, q] != 0.0:
                    out += x[p, q] * (self.E[p][q] @ v)
        return out

    def apply_hamiltonian(self, c: float, h: np.ndarray, g: np.ndarray, v: np.ndarray) -> np.ndarray:
        """H v for H = c + sum h E + 1/2 sum g (E_pq E_rs - delta_qr E_ps)."""
        n = self.n
        d = np.array([[self.E[r][s] @ v for s in range(n)] for r in range(n)])  # E_rs v
        y = np.einsum("pqrs,rsk->pqk", g, d)
        out = c * v + np.einsum("pq,pqk->k", h, d)
        out -= 0.5 * np.einsum("pqqs,psk->k", g, d)
        for p in range(n):
            for q in range(n):
                out += 0.5 * (self.E[p][q] @ y[p, q])
        return out

    def apply_cluster(self, t1: np.ndarray, t2: np.ndarray, nocc: int, v: np.ndarray) -> np.ndarray:
        """T v for T = sum t_i^a E_ai + 1/2 sum t_ij^ab E_ai E_bj (a, b counted from nocc)."""
        n = self.n
        nv = n - nocc
        d = np.array([[self.E[nocc + b][j] @ v for j in range(nocc)] for b in range(nv)])  # E_bj v
        y = 0.5 * np.einsum("ijab,bjk->aik", t2, d)
        out = np.einsum("ia,aik->k", t1, d)
        for a in range(nv):
            for i in range(nocc):
                out += self.E[nocc + a][i] @ y[a, i]
        return out

    def apply_exp_cluster(self, t1, t2, nocc: int, v: np.ndarray, sign: float) -> np.ndarray:
        """exp(sign * T) v by the terminating power series (T is nilpotent)."""
        out = v.copy()
        term = v.copy()
        for k in range(1, 4 * self.n + 2):
            term = sign * self.apply_cluster(t1, t2, nocc, term) / k
            if not np.any(term):
                break
            out += term
        return out

    def apply_hbar(self, h, g, t1, t2, nocc, v, c: float = 0.0) -> np.ndarray:
        """e^{-T} H e^{T} v, exactly."""
        u = self.apply_exp_cluster(t1, t2, nocc, v, +1.0)
        w = self.apply_hamiltonian(c, h, g, u)
        return self.apply_exp_cluster(t1, t2, nocc, w, -1.0)


# ---- single operator strings on one state (used for signs of CI coefficients) -------------

def apply_string(ops, state: int):
    """Apply a product of creation/annihilation operators to a basis state.

    `ops` is a list of ('+', P) / ('-', P) in written order (the rightmost acts first).
    Returns (coefficient, new_state); coefficient 0 when the result vanishes.
    """
    coef = 1
    s = int(state)
    for kind, P in reversed(ops):
        bit = 1 << P
        par = bin(s & (bit - 1)).count("1") & 1
        if kind == "+":
            if s & bit:
                return 0, None
            s |= bit
        else:
            if not s & bit:
                return 0, None
            s &= ~bit
        if par:
            coef = -coef
    return coef, s


@lru_cache(maxsize=None)
def cas_operators(no: int, nv: int) -> Operators:
    """E_pq on the Sz = 0 determinants of a (no, nv) active space with `no` electrons per spin."""
    return Operators(sector_basis(no + nv, no, no))
