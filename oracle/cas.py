"""One active space of the flow: its downfolded operator, Phi-dominant root and CI -> CC increment.

Passages followed:
* Eqs. (5)-(6), N = 1: the space's effective Hamiltonian is the (P + Q_int) projection of the
  dressed operator.  With the SES-CC dressing the projection of H-bar_<=2 onto the space's
  determinants (inactive occupied doubly occupied, external virtuals empty) only sees the
  normal-ordered terms whose indices are all active; rewriting them relative to the
  space's own vacuum gives E_core + sum h E + 1/2 sum W e over the active orbitals.
* The paper's solver (VQE-UCCSD) is replaced by the exact root: the eigenvector with the
  largest |overlap| with Phi, normalised so that its Phi coefficient is 1.
* "Parameters are matched to the amplitude list": the singles and doubles cluster
  amplitudes of that root (C1 = t1, C2 = t2 + t1^2/2) are the increment added to the
  pool's internal amplitudes.

Determinants of a space with no occupied and nv virtual orbitals: local orbitals
0..no-1 (occupied, ascending absolute index) then no..no+nv-1 (virtual); `no` alpha and
`no` beta electrons; kets are alpha creators (ascending) left of beta creators.

Parity pins: T = 0 limit equals frozen-core CASCI rows/columns of the full FCI matrix,
full-space case equals FCI, CI -> CC extraction inverts e^{T_int} Phi exactly,
dense eigen-solver = ``scipy.linalg.eig`` (tests).
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
import scipy.sparse as sp

from .secondq import apply_string, cas_operators, reference_state

ROOT_MIN_C0 = 1e-3


def unnormal_order(e0: float, f_act: np.ndarray, w_act: np.ndarray, nocc_act: int):
    """Rewrite E0 + F{E} + 1/2 W{e} (normal order w.r.t. the active occupied set) in
    vacuum order: h = F - sum_k (2 W_pqkk - W_pkkq), c = E0 - sum_k (h_kk + F_kk)."""
    h = f_act.copy()
    for k in range(nocc_act):
        h -= 2.0 * w_act[:, :, k, k] - w_act[:, k, k, :]
    c = e0
    for k in range(nocc_act):
        c -= h[k, k] + f_act[k, k]
    return c, h


@lru_cache(maxsize=None)
def coupling(no: int, nv: int):
    """Sparse maps from flattened (h, W) to the flattened determinant matrix."""
    ops = cas_operators(no, nv)
    dim, m = ops.basis.dim, no + nv
    E = ops.E
    rows1, cols1, vals1 = [], [], []
    for p in range(m):
        for q in range(m):
            coo = E[p][q].tocoo()
            rows1.append(coo.row * dim + coo.col)
            cols1.append(np.full(coo.nnz, p * m + q))
            vals1.append(coo.data)
    one = sp.csr_matrix((np.concatenate(vals1), (np.concatenate(rows1), np.concatenate(cols1))),
                        shape=(dim * dim, m * m))
    rows2, cols2, vals2 = [], [], []
    for p in range(m):
        for q in range(m):
            for r in range(m):
                for s in range(m):
                    op = E[p][q] @ E[r][s]
                    if q == r:
                        op = op - E[p][s]
                    coo = sp.coo_matrix(op)
                    coo.eliminate_zeros()
                    rows2.append(coo.row * dim + coo.col)
                    cols2.append(np.full(coo.nnz, ((p * m + q) * m + r) * m + s))
                    vals2.append(coo.data)
    two = sp.csr_matrix((np.concatenate(vals2), (np.concatenate(rows2), np.concatenate(cols2))),
                        shape=(dim * dim, m ** 4))
    phi = int(ops.basis.index(reference_state(m, no)))
    return one, two, dim, phi


def cas_matrix(no: int, nv: int, c: float, h: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Dense determinant matrix of c + sum h E + 1/2 sum w (E E - delta E) on the space."""
    one, two, dim, _ = coupling(no, nv)
    flat = one @ h.ravel() + 0.5 * (two @ w.ravel())
    mat = flat.reshape(dim, dim)
    mat[np.diag_indices(dim)] += c
    return mat


def phi_root(mat: np.ndarray, phi: int):
    """Eigenpair with the largest |Phi component|; returns (E, c with c[phi] = 1, status).

    status 0 = ok, 1 = selected root complex or |c_Phi| < ROOT_MIN_C0 (unit-norm vector).
    """
    w, v = np.linalg.eig(mat)
    k = int(np.argmax(np.abs(v[phi, :])))
    status = 0
    if abs(w[k].imag) > 1e-10 * max(1.0, abs(w[k].real)) or abs(v[phi, k]) < ROOT_MIN_C0:
        status = 1
    vec = (v[:, k] / v[phi, k]).real
    return float(w[k].real), vec, status


@lru_cache(maxsize=None)
def extraction_maps(no: int, nv: int):
    """Determinant index and sign of the alpha/beta singles and alpha-beta doubles of Phi."""
    ops = cas_operators(no, nv)
    m = no + nv
    phi = reference_state(m, no)
    idx = ops.basis.index

    def det(opslist):
        coef, s = apply_string(opslist, phi)
        return int(idx(s)), float(coef)

    sa = np.zeros((no, nv, 2))
    sb = np.zeros((no, nv, 2))
    dab = np.zeros((no, no, nv, nv, 2))
    for i in range(no):
        for a in range(nv):
            A = no + a
            sa[i, a] = det([("+", A), ("-", i)])
            sb[i, a] = det([("+", A + m), ("-", i + m)])
            for j in range(no):
                for b in range(nv):
                    B = no + b
                    dab[i, j, a, b] = det([("+", A), ("+", B + m), ("-", j + m), ("-", i)])
    return sa, sb, dab


def increment(no: int, nv: int, vec: np.ndarray):
    """X1[i,a] = C1, X2[i,j,a,b] = C2 - C1 C1 of a CI vector with Phi coefficient 1.

    Singles are the mean of the alpha and beta coefficients, doubles are symmetrised over
    (i a) <-> (j b); both are equalities for a spin-adapted (singlet) root.
    """
    sa, sb, dab = extraction_maps(no, nv)
    ca = vec[sa[..., 0].astype(int)] * sa[..., 1]
    cb = vec[sb[..., 0].astype(int)] * sb[..., 1]
    x1 = 0.5 * (ca + cb)
    cab = vec[dab[..., 0].astype(int)] * dab[..., 1]
    x2 = cab - np.einsum("ia,jb->ijab", x1, x1)
    x2 = 0.5 * (x2 + x2.transpose(1, 0, 3, 2))
    return x1, x2


def space_problem(e0: float, F: np.ndarray, W: np.ndarray, occ, vir):
    """(c, h, w) of one space from the global dressed integrals (absolute orbital indices)."""
    orb = list(occ) + list(vir)
    fa = F[np.ix_(orb, orb)]
    wa = W[np.ix_(orb, orb, orb, orb)]
    c, h = unnormal_order(e0, fa, wa, len(occ))
    return c, h, wa


def solve_space(e0: float, F: np.ndarray, W: np.ndarray, occ, vir):
    """Energy, increment (X1, X2) and status of one space."""
    no, nv = len(occ), len(vir)
    c, h, w = space_problem(e0, F, W, occ, vir)
    mat = cas_matrix(no, nv, c, h, w)
    _, _, _, phi = coupling(no, nv)
    e, vec, status = phi_root(mat, phi)
    x1, x2 = increment(no, nv, vec)
    return e, x1, x2, status


def solve_problem(no: int, nv: int, c: float, h: np.ndarray, w: np.ndarray):
    """Energy, increment and status of one space given its folded (c, h, w) block."""
    mat = cas_matrix(no, nv, c, h, w)
    _, _, _, phi = coupling(no, nv)
    e, vec, status = phi_root(mat, phi)
    x1, x2 = increment(no, nv, vec)
    return e, x1, x2, status
