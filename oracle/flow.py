"""The flow itself: space ordering, amplitude ownership, Jacobi sweeps, mean energy, DIIS.

Passages followed:
* Algorithm 1, final sort: spaces are ordered by ascending Delta-eps = sum eps_v - sum eps_o.
* Numerical Implementation: each amplitude is assigned to the first space (in that order)
  that can reach it, so it is updated exactly once per cycle.
* The global pool starts empty (first spaces see the bare Hamiltonian) and sweeps end
  with a barrier; they repeat until convergence.
* Results: the reported QFlow energy is the mean of the space energies E(i).

Readings where the paper is silent: ties in Delta-eps are broken by (size class, occupied
tuple, virtual tuple, input position); a t2 amplitude is reachable when both occupied and
both virtual indices are active, t2[i,j,a,b] and t2[j,i,b,a] being one amplitude; all
spaces of a sweep read the pool of the previous barrier (Jacobi); unowned amplitudes keep
their value; convergence is |dE| < 1e-8 Eh and max|dt| < 1e-7.
"""
from __future__ import annotations

import numpy as np

from . import cas, hbar
from .ccsd import Diis, fock_diagonal


def space_orbitals(row):
    no, nv = int(row[0]), int(row[1])
    orb = [int(x) for x in row[2:2 + no + nv]]
    return orb[:no], orb[no:]


def delta_eps(row, eps: np.ndarray) -> float:
    """sum eps_v - sum eps_o, each sum taken in ascending index order."""
    occ, vir = space_orbitals(row)
    sv = 0.0
    for a in vir:
        sv = sv + float(eps[a])
    so = 0.0
    for i in occ:
        so = so + float(eps[i])
    return sv - so


def sort_spaces(spaces: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """Permutation: sorted position -> input index."""
    keys = []
    for k, row in enumerate(spaces):
        occ, vir = space_orbitals(row)
        keys.append((delta_eps(row, eps), int(row[0]), tuple(occ), tuple(vir), k))
    keys.sort()
    return np.array([k[-1] for k in keys], dtype=np.int64)


def owner_maps(spaces_sorted: np.ndarray, nocc: int, nvir: int):
    """owner1[i,a], owner2[i,j,a,b]: sorted index of the first space reaching the amplitude, or -1."""
    own1 = np.full((nocc, nvir), -1, dtype=np.int64)
    own2 = np.full((nocc, nocc, nvir, nvir), -1, dtype=np.int64)
    for s, row in enumerate(spaces_sorted):
        occ, vir = space_orbitals(row)
        va = [a - nocc for a in vir]
        for i in occ:
            for a in va:
                if own1[i, a] < 0:
                    own1[i, a] = s
        for i in occ:
            for j in occ:
                for a in va:
                    for b in va:
                        if own2[i, j, a, b] < 0:
                            own2[i, j, a, b] = s
                            own2[j, i, b, a] = s
    return own1, own2


def solve_all(e0, F, W, spaces_sorted, pool=None):
    """Per-space (E, X1, X2, status) for every space of the sorted list."""
    jobs = [space_orbitals(row) for row in spaces_sorted]
    if pool is None:
        return [cas.solve_space(e0, F, W, occ, vir) for occ, vir in jobs]
    return pool.starmap(cas.solve_space, [(e0, F, W, occ, vir) for occ, vir in jobs], chunksize=16)


def merge(t1, t2, spaces_sorted, results, own1, own2, nocc):
    """t_new[x] = t_old[x] + X_owner(x)[x]; unowned amplitudes unchanged.  A space whose root
    is flagged (status != 0: complex, or |c_Phi| below the limit) has no usable increment, so
    the amplitudes it owns keep their value as well."""
    t1n, t2n = t1.copy(), t2.copy()
    for s, (row, res) in enumerate(zip(spaces_sorted, results)):
        occ, vir = space_orbitals(row)
        va = [a - nocc for a in vir]
        _, x1, x2, st = res
        if st != 0:
            continue
        for ii, i in enumerate(occ):
            for aa, a in enumerate(va):
                if own1[i, a] == s:
                    t1n[i, a] = t1[i, a] + x1[ii, aa]
            for jj, j in enumerate(occ):
                for aa, a in enumerate(va):
                    for bb, b in enumerate(va):
                        if own2[i, j, a, b] == s:
                            t2n[i, j, a, b] = t2[i, j, a, b] + x2[ii, jj, aa, bb]
    return t1n, t2n


class Flow:
    """Plain FP64 QFlow in the SES-CC reading, Jacobi sweeps from an empty pool."""

    def __init__(self, h, g, nocc, spaces, t1=None, t2=None, diis: bool = False, pool=None):
        self.h, self.g, self.nocc = h, g, nocc
        n = h.shape[0]
        self.nvir = n - nocc
        self.eps = fock_diagonal(h, g, nocc)
        self.perm = sort_spaces(spaces, self.eps)
        self.spaces = np.asarray(spaces)[self.perm]
        self.own1, self.own2 = owner_maps(self.spaces, nocc, self.nvir)
        self.t1 = np.zeros((nocc, self.nvir)) if t1 is None else t1.copy()
        self.t2 = np.zeros((nocc, nocc, self.nvir, self.nvir)) if t2 is None else t2.copy()
        self.e_mean = None
        self.energies = None
        self.diis = Diis() if diis else None
        self.pool = pool

    def uncovered(self) -> int:
        return int((self.own1 < 0).sum() + (self.own2 < 0).sum())

    def dress(self):
        return hbar.hbar2(self.h, self.g, self.t1, self.t2, self.nocc)

    def sweep(self):
        """One barrier-to-barrier sweep; returns (E_mean, dE, max|dt|, n_failed)."""
        e0, F, W = self.dress()
        res = solve_all(e0, F, W, self.spaces, self.pool)
        t1n, t2n = merge(self.t1, self.t2, self.spaces, res, self.own1, self.own2, self.nocc)
        if self.diis is not None:
            vec = np.concatenate([t1n.ravel(), t2n.ravel()])
            err = np.concatenate([(t1n - self.t1).ravel(), (t2n - self.t2).ravel()])
            vec = self.diis.push(vec, err)
            t1n = vec[:self.t1.size].reshape(self.t1.shape)
            t2n = vec[self.t1.size:].reshape(self.t2.shape)
        dt = max(np.abs(t1n - self.t1).max(initial=0.0), np.abs(t2n - self.t2).max(initial=0.0))
        self.t1, self.t2 = t1n, t2n
        self.energies = np.array([r[0] for r in res])
        e_mean = float(np.mean(self.energies))
        de = float("inf") if self.e_mean is None else e_mean - self.e_mean
        self.e_mean = e_mean
        nfail = int(sum(r[3] != 0 for r in res))
        return e_mean, de, float(dt), nfail

    def sweep_waves(self, wave: int):
        """One sweep in waves of `wave` spaces in Delta-eps order (Numerical Implementation: the
        pool is populated progressively as spaces are traversed; process groups take the spaces
        in list order, so the spaces running together see the same pool).  Each wave is
        downfolded with the pool left by the waves before it, and its owned amplitudes are updated
        before the next wave starts.  wave >= nspaces is the Jacobi sweep.  Returns what sweep()
        returns; max|dt| is taken over the whole sweep and DIIS (if on) acts on the sweep's start
        and end pools."""
        if wave < 1:
            raise ValueError("wave must be >= 1")
        t1s, t2s = self.t1, self.t2
        t1c, t2c = t1s.copy(), t2s.copy()
        ns = len(self.spaces)
        energies = np.zeros(ns)
        status = np.zeros(ns, dtype=int)
        for lo in range(0, ns, wave):
            hi = min(ns, lo + wave)
            e0, F, W = hbar.hbar2(self.h, self.g, t1c, t2c, self.nocc)
            res = solve_all(e0, F, W, self.spaces[lo:hi], self.pool)
            for s, (row, r) in enumerate(zip(self.spaces[lo:hi], res), start=lo):
                occ, vir = space_orbitals(row)
                va = [a - self.nocc for a in vir]
                energies[s], x1, x2, status[s] = r
                if status[s] != 0:  # a flagged root leaves its owned amplitudes unchanged
                    continue
                for ii, i in enumerate(occ):
                    for aa, a in enumerate(va):
                        if self.own1[i, a] == s:
                            t1c[i, a] = t1c[i, a] + x1[ii, aa]
                    for jj, j in enumerate(occ):
                        for aa, a in enumerate(va):
                            for bb, b in enumerate(va):
                                if self.own2[i, j, a, b] == s:
                                    t2c[i, j, a, b] = t2c[i, j, a, b] + x2[ii, jj, aa, bb]
        t1n, t2n = t1c, t2c
        if self.diis is not None:
            vec = np.concatenate([t1n.ravel(), t2n.ravel()])
            err = np.concatenate([(t1n - t1s).ravel(), (t2n - t2s).ravel()])
            vec = self.diis.push(vec, err)
            t1n = vec[:t1s.size].reshape(t1s.shape)
            t2n = vec[t1s.size:].reshape(t2s.shape)
        dt = max(np.abs(t1n - t1s).max(initial=0.0), np.abs(t2n - t2s).max(initial=0.0))
        self.t1, self.t2 = t1n, t2n
        self.energies = energies
        e_mean = float(np.mean(energies))
        de = float("inf") if self.e_mean is None else e_mean - self.e_mean
        self.e_mean = e_mean
        return e_mean, de, float(dt), int((status != 0).sum())

    def run(self, tol_e: float = 1e-8, tol_t: float = 1e-7, max_sweeps: int = 100):
        hist = []
        for _ in range(max_sweeps):
            e, de, dt, nf = self.sweep()
            hist.append((e, de, dt, nf))
            if abs(de) < tol_e and dt < tol_t:
                break
        return hist


# ---- counts the paper prints (Results, Table I, abstract) ------------------------------------

def qubits(no: int, nv: int) -> int:
    """Qubits of a problem with no occupied and nv virtual spatial orbitals: 2 (no + nv)."""
    return 2 * (no + nv)


def minimal_coverage_size(no: int, nv: int) -> int:
    """|C_min| = C(No, 2) C(Nv, 2) (the (o1<o2, v1<v2) tuples of Algorithm 1)."""
    from math import comb
    return comb(no, 2) * comb(nv, 2)


def spin_orbital_parameters(no: int, nv: int) -> int:
    """Unique spin-conserving singles and doubles amplitudes over spin orbitals."""
    from math import comb
    return 2 * no * nv + 2 * comb(no, 2) * comb(nv, 2) + (no * nv) ** 2


def spatial_parameters(no: int, nv: int) -> int:
    """Unique closed-shell amplitudes: t1[i,a] plus t2[i,j,a,b] ~ t2[j,i,b,a]."""
    ov = no * nv
    return ov + ov * (ov + 1) // 2
