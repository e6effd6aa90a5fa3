"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module draws random numbers and builds the *inputs* of a Quantum Flow run:
orbital energies, molecular-orbital integrals shaped like a density-fitted closed-shell
RHF system, and active-space lists.  It holds none of the flow's own arithmetic
(no dressing, no CAS solve, no amplitude update) and imports nothing from the
rest of the package, so both sides of every parity test can use it.

Integral recipe (the paper's molecules are not available, so this stands in for them):
  * occupied orbital energies  eps_i ~ U[-1.5, -0.5] Eh, virtual eps_a ~ U[0.2, 3.0] Eh,
    each group sorted ascending, occupied first;
  * (pq|rs) = sum_{L < 2n} B^L_pq B^L_rs with B^L symmetric, upper triangle (p <= q) drawn
    in (L, p, q) order, entries N(0,1) * 0.3 * exp(-|p-q|/xi) / sqrt(2n);
  * h_pq = eps_p delta_pq - sum_i [2 (pq|ii) - (pi|iq)], so that the closed-shell Fock
    matrix of the lowest `nocc` orbitals is diag(eps) and the reference determinant is a
    canonical RHF determinant; no nuclear repulsion.

Active spaces follow the paper's (n_o, n_v) notation (Algorithm 1 input): a space is a
set of n_o occupied and n_v virtual orbitals, stored as a row of the int32 array
``spaces[k] = (n_o, n_v, orb[0..5])`` with the occupied indices first, each group
ascending, unused slots = -1.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

SPACE_FIELDS = 8  # n_o, n_v, orb[6]


@dataclass(frozen=True)
class SystemSpec:
    name: str
    n: int          # spatial orbitals
    nocc: int       # doubly occupied orbitals
    xi: float       # decay length of the density-fitting factors
    seed: int       # integral seed
    space_mode: str  # "all33" | "mixed" | "sample33"
    space_seed: int = 0
    n_spaces: int = 0        # per size class for "mixed", total for "sample33"


# The five synthetic systems: 10, 24, 40, 82 and 114 orbitals.  The two largest keep the
# orbital counts of the paper's propane cc-pVDZ (82) and H2O cc-pVQZ (114) parent problems.
SYSTEMS = {
    "n10": SystemSpec("n10", 10, 3, 3.0, 0, "all33"),
    "n24": SystemSpec("n24", 24, 5, 4.0, 1, "all33"),
    "n40": SystemSpec("n40", 40, 6, 4.0, 2, "mixed", space_seed=3, n_spaces=20000),
    "n82": SystemSpec("n82", 82, 10, 5.0, 3, "all33"),
    "n114": SystemSpec("n114", 114, 11, 8.0, 4, "sample33", space_seed=5, n_spaces=2000000),
}


def orbital_energies(rng: np.random.Generator, n: int, nocc: int) -> np.ndarray:
    eo = np.sort(rng.uniform(-1.5, -0.5, size=nocc))
    ev = np.sort(rng.uniform(0.2, 3.0, size=n - nocc))
    return np.concatenate([eo, ev])


def df_factors(rng: np.random.Generator, n: int, xi: float) -> np.ndarray:
    """B[L, p, q], symmetric in (p, q), L < 2n."""
    nl = 2 * n
    iu, ju = np.triu_indices(n)
    z = rng.standard_normal((nl, iu.size))
    scale = 0.3 * np.exp(-np.abs(iu - ju) / xi) / math.sqrt(nl)
    b = np.zeros((nl, n, n))
    b[:, iu, ju] = z * scale
    b[:, ju, iu] = z * scale
    return b


def make_system(n: int, nocc: int, xi: float, seed: int):
    """Return (eps, h, eri) in float64; eri[p,q,r,s] = (pq|rs) (chemists' notation)."""
    rng = np.random.default_rng(seed)
    eps = orbital_energies(rng, n, nocc)
    b = df_factors(rng, n, xi)
    bm = b.reshape(2 * n, n * n)
    eri = (bm.T @ bm).reshape(n, n, n, n)
    occ = np.arange(nocc)
    j = eri[:, :, occ, occ].sum(axis=2)              # sum_i (pq|ii)
    k = eri[:, occ, occ, :].sum(axis=1)              # sum_i (pi|iq)
    h = np.diag(eps) - (2.0 * j - k)
    h = 0.5 * (h + h.T)
    return eps, np.ascontiguousarray(h), np.ascontiguousarray(eri)


def _space_row(occ, vir):
    row = np.full(SPACE_FIELDS, -1, dtype=np.int32)
    row[0], row[1] = len(occ), len(vir)
    row[2:2 + len(occ)] = occ
    row[2 + len(occ):2 + len(occ) + len(vir)] = vir
    return row


def all_spaces(n: int, nocc: int, no: int = 3, nv: int = 3) -> np.ndarray:
    """Every (no, nv) space, occupied tuple major, virtual tuple minor (lexicographic)."""
    occ_t = np.array(list(itertools.combinations(range(nocc), no)), dtype=np.int32).reshape(-1, no)
    vir_t = np.array(list(itertools.combinations(range(nocc, n), nv)), dtype=np.int32).reshape(-1, nv)
    out = np.full((len(occ_t) * len(vir_t), SPACE_FIELDS), -1, dtype=np.int32)
    out[:, 0], out[:, 1] = no, nv
    out[:, 2:2 + no] = np.repeat(occ_t, len(vir_t), axis=0)
    out[:, 2 + no:2 + no + nv] = np.tile(vir_t, (len(occ_t), 1))
    return out


def _unrank_combination(rank: np.ndarray, m: int, k: int) -> np.ndarray:
    """Lexicographic unranking of k-subsets of range(m) (vectorised over ranks)."""
    rank = np.asarray(rank, dtype=np.int64).copy()
    out = np.empty((rank.size, k), dtype=np.int32)
    start = np.zeros(rank.size, dtype=np.int64)
    for pos in range(k):
        rem = k - pos - 1
        c = start.copy()
        while True:
            cnt = _comb_vec(m - c - 1, rem)   # subsets whose element at `pos` is c
            adv = (rank >= cnt) & (c < m)
            if not adv.any():
                break
            rank = np.where(adv, rank - cnt, rank)
            c = np.where(adv, c + 1, c)
        out[:, pos] = c
        start = c + 1
    return out


def _comb_vec(a: np.ndarray, r: int) -> np.ndarray:
    a = a.astype(np.int64)
    res = np.ones_like(a)
    for t in range(r):
        res = res * (a - t)
    res //= math.factorial(r)
    return np.where(a >= r, res, 0)


def sampled_spaces(n: int, nocc: int, count: int, seed: int, no: int = 3, nv: int = 3) -> np.ndarray:
    """`count` distinct (no, nv) spaces drawn uniformly without replacement."""
    nvir = n - nocc
    c_o, c_v = math.comb(nocc, no), math.comb(nvir, nv)
    rng = np.random.default_rng(seed)
    picks = rng.choice(c_o * c_v, size=count, replace=False)
    oi, vi = np.divmod(picks, c_v)
    occ = _unrank_combination(oi, nocc, no)
    vir = _unrank_combination(vi, nvir, nv) + nocc
    out = np.full((count, SPACE_FIELDS), -1, dtype=np.int32)
    out[:, 0], out[:, 1] = no, nv
    out[:, 2:2 + no] = occ
    out[:, 2 + no:2 + no + nv] = vir
    return out


def mixed_spaces(n: int, nocc: int, per_class: int, seed: int) -> np.ndarray:
    """`per_class` spaces of each size (1,1), (2,2), (3,3).

    (1,1) and (2,2) are drawn uniformly with replacement (there are fewer distinct ones than
    requested), (3,3) uniformly without replacement.  Classes are concatenated in this order.
    """
    rng = np.random.default_rng(seed)
    nvir = n - nocc
    rows = []
    for k in (1, 2):
        c_o, c_v = math.comb(nocc, k), math.comb(nvir, k)
        picks = rng.integers(0, c_o * c_v, size=per_class)
        oi, vi = np.divmod(picks, c_v)
        occ = _unrank_combination(oi, nocc, k)
        vir = _unrank_combination(vi, nvir, k) + nocc
        blk = np.full((per_class, SPACE_FIELDS), -1, dtype=np.int32)
        blk[:, 0], blk[:, 1] = k, k
        blk[:, 2:2 + k] = occ
        blk[:, 2 + k:2 + 2 * k] = vir
        rows.append(blk)
    c_o, c_v = math.comb(nocc, 3), math.comb(nvir, 3)
    picks = rng.choice(c_o * c_v, size=per_class, replace=False)
    oi, vi = np.divmod(picks, c_v)
    blk = np.full((per_class, SPACE_FIELDS), -1, dtype=np.int32)
    blk[:, 0], blk[:, 1] = 3, 3
    blk[:, 2:5] = _unrank_combination(oi, nocc, 3)
    blk[:, 5:8] = _unrank_combination(vi, nvir, 3) + nocc
    rows.append(blk)
    return np.concatenate(rows)


def system_inputs(name: str, with_spaces: bool = True):
    """(eps, h, eri, spaces) for one of the named synthetic systems."""
    s = SYSTEMS[name]
    eps, h, eri = make_system(s.n, s.nocc, s.xi, s.seed)
    if not with_spaces:
        return eps, h, eri, None
    if s.space_mode == "all33":
        sp = all_spaces(s.n, s.nocc)
    elif s.space_mode == "mixed":
        sp = mixed_spaces(s.n, s.nocc, s.n_spaces, s.space_seed)
    else:
        sp = sampled_spaces(s.n, s.nocc, s.n_spaces, s.space_seed)
    return eps, h, eri, sp


def random_amplitudes(nocc: int, nvir: int, seed: int, scale1: float = 0.02, scale2: float = 0.03):
    """Seeded closed-shell test amplitudes t1[i,a], t2[i,j,a,b] with t2[i,j,a,b] = t2[j,i,b,a]."""
    rng = np.random.default_rng(seed)
    t1 = scale1 * rng.standard_normal((nocc, nvir))
    t2 = scale2 * rng.standard_normal((nocc, nocc, nvir, nvir))
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    return t1, t2


# ---- warm-start network inputs -----------------------------------------------------------------

def mlp_init_params(n_in: int, hidden: int, n_out: int, seed: int) -> np.ndarray:
    """Seeded Glorot-uniform weights and zero biases, packed W1, b1, W2, b2, W3, b3 with every W
    stored [fan_in][fan_out] row-major (float64; callers cast)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fi, fo in ((n_in, hidden), (hidden, hidden), (hidden, n_out)):
        lim = math.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-lim, lim, size=fi * fo))
        parts.append(np.zeros(fo))
    return np.concatenate(parts)


def mlp_init_model(hidden: int, seed: int, n_in: int = 708, n_out: int = 54) -> np.ndarray:
    """Initial model of the 6e6o warm-start network: parameters followed by placeholder
    standardisation (mean 0, scale 1) that training replaces (float32)."""
    p = mlp_init_params(n_in, hidden, n_out, seed)
    return np.concatenate([p, np.zeros(n_in), np.ones(n_in), np.zeros(n_out), np.ones(n_out)]).astype(np.float32)
