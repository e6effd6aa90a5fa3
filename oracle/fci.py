"""Determinant full configuration interaction (the exact limit the flow is compared with).

The paper's parent problem is the full target space of Eq. (1); for tiny systems its exact
ground state is the FCI energy.  When an active space spans every orbital and the pool is
empty (first sweep), the flow's space energy must equal this number.

Dense ``numpy.linalg.eigh`` for small determinant spaces, ``scipy.sparse.linalg.eigsh``
(Lanczos) on the exact H-vector product otherwise.  Pin: the two agree on mid-size cases
(tests), and CCSD = FCI for two electrons.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .secondq import Operators, reference_state, sector_basis


def fci_energy(h: np.ndarray, g: np.ndarray, nocc: int, c: float = 0.0, dense_limit: int = 2500) -> float:
    n = h.shape[0]
    ops = Operators(sector_basis(n, nocc, nocc))
    dim = ops.basis.dim
    if dim <= dense_limit:
        hm = np.empty((dim, dim))
        eye = np.eye(dim)
        for k in range(dim):
            hm[:, k] = ops.apply_hamiltonian(c, h, g, eye[:, k])
        return float(np.linalg.eigvalsh(0.5 * (hm + hm.T))[0])
    lin = spla.LinearOperator((dim, dim), matvec=lambda x: ops.apply_hamiltonian(c, h, g, np.asarray(x).ravel()),
                              dtype=float)
    v0 = ops.basis.unit(reference_state(n, nocc))
    w = spla.eigsh(lin, k=1, which="SA", v0=v0 + 1e-3, tol=1e-13, maxiter=5000, return_eigenvectors=False)
    return float(w[0])
