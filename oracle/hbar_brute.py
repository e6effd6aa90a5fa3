"""Normal-ordered <=2-body part of e^{-T} H e^{T}, read off exact Fock-space matrix elements.

This is the *definition* of the dressed Hamiltonian used by the flow (Eqs. 5-6 with N = 1
in the SES-CC reading: H-bar = e^{-T} H e^{T}, normal ordered with respect to the closed-shell
reference Phi and truncated to one- and two-body terms), evaluated by brute force for tiny
orbital counts (2n spin orbitals, 2^{2n} Fock states).  It pins the closed-form spin-free
formulas of ``oracle.hbar``.

Method.  Relative to Phi, every a / a+ is either a quasi-particle creator (a+ on an empty
orbital, a on a filled one) or a quasi-particle annihilator.  A normal-ordered string with
creators X and annihilators Y (quasi-particle sets) connects |nu> = Phi with the Y
quasi-particles present to |mu> = Phi with the X quasi-particles present.  Between such a
pair only the components of H-bar whose quasi-particle counts fit inside (|X|, |Y|)
contribute, so with |X| + |Y| <= 4 no three-body or higher term can reach the element.
Subtracting the already-extracted lower-rank parts leaves exactly one coefficient times the
(+-1) matrix element of the string itself.

Parity pins for this module: exact by construction (definition); cross-checked in the tests
against the T = 0 limit (bare integrals) and the T1-only limit (an exact orbital
similarity transformation).
"""
from __future__ import annotations

import numpy as np

from .secondq import Operators, apply_string, fock_basis, reference_state


def _quasi_sets(ops, phi: int):
    """Split a string into quasi-particle creators X and annihilators Y; return the
    normal-ordered (creators left, stable) string and the permutation sign."""
    qc, qa = [], []
    for pos, (kind, P) in enumerate(ops):
        occupied = (phi >> P) & 1
        is_creator = (kind == "+" and not occupied) or (kind == "-" and occupied)
        (qc if is_creator else qa).append((pos, kind, P))
    order = [x[0] for x in qc] + [x[0] for x in qa]
    inv = sum(1 for i in range(len(order)) for j in range(i + 1, len(order)) if order[i] > order[j])
    sign = -1 if inv & 1 else 1
    X = [P for _, _, P in qc]
    Y = [P for _, _, P in qa]
    nops = [(k, P) for _, k, P in qc] + [(k, P) for _, k, P in qa]
    return X, Y, nops, sign


def _flip(phi: int, orbs) -> int:
    s = phi
    for P in orbs:
        s ^= 1 << P
    return s


def normal_ordered_element(ops, phi: int, mu: int, nu: int) -> float:
    """<mu| {ops} |nu> for the string normal ordered with respect to phi."""
    _, _, nops, sign = _quasi_sets(ops, phi)
    c, s = apply_string(nops, nu)
    if c == 0 or s != mu:
        return 0.0
    return float(sign * c)


class HbarBrute:
    """E0, spin-orbital fbar[P, Q] and spin-free Wbar[p, q, r, s] of e^{-T} H e^{T}."""

    def __init__(self, h, g, t1, t2, nocc: int, c: float = 0.0):
        self.n = n = h.shape[0]
        self.nocc = nocc
        self.ops = Operators(fock_basis(n))
        self.basis = self.ops.basis
        self.phi = reference_state(n, nocc)
        self._args = (h, g, t1, t2, nocc)
        self._c = c
        self._cache = {}
        self.E0 = self._elem(self.phi, self.phi)
        self.fbar = self._one_body()

    def _col(self, nu: int) -> np.ndarray:
        if nu not in self._cache:
            h, g, t1, t2, nocc = self._args
            self._cache[nu] = self.ops.apply_hbar(h, g, t1, t2, nocc, self.basis.unit(nu), c=self._c)
        return self._cache[nu]

    def _elem(self, mu: int, nu: int) -> float:
        return float(self._col(nu)[int(self.basis.index(mu))])

    def _one_body(self) -> np.ndarray:
        m = 2 * self.n
        f = np.zeros((m, m))
        for P in range(m):
            for Q in range(m):
                ops = [("+", P), ("-", Q)]
                X, Y, _, _ = _quasi_sets(ops, self.phi)
                mu, nu = _flip(self.phi, X), _flip(self.phi, Y)
                val = self._elem(mu, nu) - (self.E0 if mu == nu else 0.0)
                f[P, Q] = val / normal_ordered_element(ops, self.phi, mu, nu)
        return f

    def w_element(self, p: int, q: int, r: int, s: int) -> float:
        """Wbar_pqrs = coefficient of {a+_{p a} a+_{r b} a_{s b} a_{q a}} (spin-free, chemists' order)."""
        n = self.n
        ops = [("+", p), ("+", r + n), ("-", s + n), ("-", q)]
        X, Y, _, _ = _quasi_sets(ops, self.phi)
        mu, nu = _flip(self.phi, X), _flip(self.phi, Y)
        val = self._elem(mu, nu) - (self.E0 if mu == nu else 0.0)
        m = 2 * n
        for P in range(m):
            for Q in range(m):
                if self.fbar[P, Q] != 0.0:
                    e = normal_ordered_element([("+", P), ("-", Q)], self.phi, mu, nu)
                    if e:
                        val -= self.fbar[P, Q] * e
        return val / normal_ordered_element(ops, self.phi, mu, nu)

    def spin_free_fock(self) -> np.ndarray:
        n = self.n
        return self.fbar[:n, :n].copy()

    def wbar(self) -> np.ndarray:
        n = self.n
        w = np.zeros((n, n, n, n))
        for p in range(n):
            for q in range(n):
                for r in range(n):
                    for s in range(n):
                        w[p, q, r, s] = self.w_element(p, q, r, s)
        return w
