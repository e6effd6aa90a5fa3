"""Closed-shell MP2 and CCSD reference energies (the paper's yardstick for "% correlation").

The paper compares every QFlow energy with canonical CCSD (Results, Table I).  In the
SES-CC reading used here the CCSD amplitudes are an exact fixed point of the flow, so the
CCSD energy is also a parity target for converged sweeps.

``ccsd`` solves <S|H-bar|Phi> = <D|H-bar|Phi> = 0 with the residual blocks of
``oracle.hbar`` (Jacobi updates on orbital-energy denominators, DIIS).  Pins: the first
iteration reproduces the closed-form MP2 energy; for two electrons CCSD equals FCI; the
residuals equal determinant-space e^{-T} H e^{T} Phi (tests).
"""
from __future__ import annotations

import numpy as np

from . import hbar


def fock_diagonal(h: np.ndarray, g: np.ndarray, nocc: int) -> np.ndarray:
    """f_pp = h_pp + sum_k [2 (pp|kk) - (pk|kp)], summed k = 0, 1, ... in that order."""
    n = h.shape[0]
    out = np.empty(n)
    for p in range(n):
        acc = float(h[p, p])
        for k in range(nocc):
            acc = acc + (2.0 * float(g[p, p, k, k]) - float(g[p, k, k, p]))
        out[p] = acc
    return out


def mp2_energy(eps: np.ndarray, g: np.ndarray, nocc: int) -> float:
    """E_MP2 = sum (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b) (canonical RHF)."""
    o, v = slice(0, nocc), slice(nocc, g.shape[0])
    ovov = g[o, v, o, v]
    eo, ev = eps[o], eps[v]
    d = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    return float(np.sum(ovov * (2.0 * ovov - ovov.transpose(0, 3, 2, 1)) / d))


def hf_energy(h: np.ndarray, g: np.ndarray, nocc: int) -> float:
    o = slice(0, nocc)
    return float(2.0 * np.trace(h[o, o]) + 2.0 * np.einsum("kkll->", g[o, o, o, o])
                 - np.einsum("kllk->", g[o, o, o, o]))


def residuals(h, g, t1, t2, nocc):
    """(E0, R1[i,a], R2[i,j,a,b]) = (<Phi|H-bar|Phi>, <S|H-bar|Phi>, <D|H-bar|Phi>)."""
    ht, gt = hbar.t1_transform(h, g, t1, nocc)
    _, f = hbar.reference_terms(ht, gt, nocc)
    e0 = hbar.energy(ht, gt, t2, nocc)
    r1 = hbar.singles_residual(f, gt, t2, nocc).T
    r2 = hbar.doubles_residual(f, gt, t2, nocc)
    return e0, r1, r2


class Diis:
    """Pulay DIIS on a flat vector with error vectors; plain least squares with a Lagrange row."""

    def __init__(self, size: int = 8):
        self.size = size
        self.vecs, self.errs = [], []

    def push(self, vec: np.ndarray, err: np.ndarray) -> np.ndarray:
        self.vecs.append(vec.copy())
        self.errs.append(err.copy())
        if len(self.vecs) > self.size:
            self.vecs.pop(0)
            self.errs.pop(0)
        m = len(self.vecs)
        if m < 2:
            return vec
        b = np.empty((m + 1, m + 1))
        b[:m, :m] = [[float(ei @ ej) for ej in self.errs] for ei in self.errs]
        b[m, :m] = b[:m, m] = -1.0
        b[m, m] = 0.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        try:
            c = np.linalg.solve(b, rhs)
        except np.linalg.LinAlgError:
            return vec
        return sum(ci * vi for ci, vi in zip(c[:m], self.vecs))


def ccsd(h, g, nocc, tol: float = 1e-11, max_iter: int = 200, diis: bool = True, t1=None, t2=None):
    """Closed-shell CCSD; returns (E_CCSD, t1, t2, iterations)."""
    n = h.shape[0]
    nv = n - nocc
    eps = fock_diagonal(h, g, nocc)
    eo, ev = eps[:nocc], eps[nocc:]
    d1 = eo[:, None] - ev[None, :]
    d2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    t1 = np.zeros((nocc, nv)) if t1 is None else t1.copy()
    t2 = np.zeros((nocc, nocc, nv, nv)) if t2 is None else t2.copy()
    acc = Diis() if diis else None
    e_old = 0.0
    for it in range(1, max_iter + 1):
        e0, r1, r2 = residuals(h, g, t1, t2, nocc)
        t1n = t1 + r1 / d1
        t2n = t2 + r2 / d2
        t2n = 0.5 * (t2n + t2n.transpose(1, 0, 3, 2))
        if acc is not None:
            vec = np.concatenate([t1n.ravel(), t2n.ravel()])
            err = np.concatenate([(t1n - t1).ravel(), (t2n - t2).ravel()])
            vec = acc.push(vec, err)
            t1n = vec[:t1.size].reshape(t1.shape)
            t2n = vec[t1.size:].reshape(t2.shape)
        dt = max(np.abs(t1n - t1).max(initial=0.0), np.abs(t2n - t2).max(initial=0.0))
        t1, t2 = t1n, t2n
        if max(np.abs(r1).max(initial=0.0), np.abs(r2).max(initial=0.0)) < tol and abs(e0 - e_old) < tol:
            e0, _, _ = residuals(h, g, t1, t2, nocc)
            return float(e0), t1, t2, it
        e_old = e0
        if dt == 0.0 and it > 1:
            break
    e0, r1, r2 = residuals(h, g, t1, t2, nocc)
    return float(e0), t1, t2, max_iter
