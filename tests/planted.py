"""Hand-built dressed Hamiltonians that exercise the root selection of a space's solver.

* ``complex_pair(k)``: one (k, k) space on 2k orbitals whose Phi-dominant root is one of a
  complex pair.  F is diagonal with the virtual energies summing to the occupied ones, so the
  doubles (i j -> a b) are degenerate with Phi, and W holds only a non-symmetric pair of couplings
  between Phi and them, <D|H|Phi> = -y (elements W_aibj) and <Phi|H|D> = +x (W_iajb): the block
  [[0, x], [-y, 0]] has the eigenvalues +-i sqrt(xy).  For k >= 2 the same couplings lead on to
  the quadruple (i i j j -> a a b b), also degenerate; the on-site terms W_aaaa = W_bbbb = U lift
  it (and only it: a and b are never doubly occupied elsewhere in the chain), so the pair stays
  the Phi-dominant root.  Everything else is uncoupled.
* ``lowered_virtual(h, g, nocc)``: the bare Hamiltonian (T = 0) of a system with the first
  virtual orbital energy moved below the highest occupied one, so that in every space holding both
  orbitals the double excitation between them sits far below Phi and the lowest root is not the
  Phi-dominant one.
"""
import numpy as np


def complex_pair(k: int, x: float = 0.04, y: float = 0.03):
    n = 2 * k
    eo = -0.9 + 0.2 * np.arange(k)           # occupied energies
    ev = eo[::-1] + 0.0                       # virtual energies: same multiset, so sums match
    ev = np.sort(ev)
    F = np.diag(np.concatenate([eo, ev]))
    W = np.zeros((n,) * 4)
    i, j = 0, k - 1                           # occupied pair (i = j for k = 1)
    a, b = k + 0, k + k - 1                   # virtual pair with e_a + e_b = e_i + e_j
    assert abs(ev[0] + ev[k - 1] - eo[0] - eo[k - 1]) < 1e-15
    planted = [((a, i, b, j), -y), ((i, a, j, b), x)]
    if k >= 2:  # (for k = 1 the double itself is the top of the chain)
        planted += [((a, a, a, a), 2.0), ((b, b, b, b), 2.0)]
    for (p, q, r, s), v in planted:
        W[p, q, r, s] = v
        W[r, s, p, q] = v                     # pair symmetry W_pqrs = W_rspq
    e0 = 2.0 * eo.sum()
    space = np.array([[k, k] + list(range(n)) + [-1] * (6 - n)], dtype=np.int32)
    return n, k, e0, F, W, space


def lowered_virtual(h, g, nocc: int, shift: float = 0.35):
    from oracle import ccsd
    F = h + 2.0 * np.einsum("pqkk->pq", g[:, :, :nocc, :nocc]) - np.einsum("pkkq->pq", g[:, :nocc, :nocc, :])
    F = F.copy()
    F[nocc, nocc] = F[nocc - 1, nocc - 1] - shift
    return ccsd.hf_energy(h, g, nocc), F, g.copy()


def selected_is_lowest(e0, F, W, occ, vir) -> bool:
    """Whether the oracle's selected (Phi-dominant) root is the lowest real eigenvalue."""
    from oracle import cas
    no, nv = len(occ), len(vir)
    c, hh, w = cas.space_problem(e0, F, W, occ, vir)
    mat = cas.cas_matrix(no, nv, c, hh, w)
    ev = np.linalg.eigvals(mat)
    e_sel, _, _, st = cas.solve_space(e0, F, W, occ, vir)
    lowest = ev.real[np.abs(ev.imag) < 1e-10].min()
    return abs(e_sel - lowest) < 1e-9
