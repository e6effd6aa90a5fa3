"""Coverage-driven active-space sampling (Numerical Implementation, Algorithm 1).

Test infrastructure only: the library's host sampler is checked against this module.

The algorithm: the minimal coverage set holds every (o1 < o2, v1 < v2) tuple of occupied and
virtual orbitals.  Candidates draw n_o occupied and n_v virtual orbitals uniformly without
replacement; a candidate that covers at least one tuple not yet covered is kept (with its
Delta-eps = sum eps_v - sum eps_o) and its tuples leave the remaining set; candidates that add
nothing are discarded.  When nothing remains, the kept spaces are sorted by ascending Delta-eps.

Readings where the paper is silent (the random numbers are not specified, only "a fixed seed"):
* generator: SplitMix64 (Steele, Lea and Flood, 2014): the state advances by 0x9E3779B97F4A7C15
  and each output is the state passed through the mixing function
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB; z ^ (z >> 31);
  the seed is the initial state;
* a draw of k of m elements is a partial Fisher-Yates shuffle of 0..m-1 (restarted from the
  identity for every draw): for i < k, swap element i with element i + (u mod (m - i)), u the next
  output; the k leading elements, sorted, are the draw; occupied orbitals are drawn first;
* Delta-eps sums each part in ascending orbital order; the final sort is stable (ties keep the
  order in which the spaces were kept).
"""
from __future__ import annotations

import math

import numpy as np

MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        return z ^ (z >> 31)


def draw(rng: SplitMix64, m: int, k: int) -> list[int]:
    """k distinct elements of 0..m-1, ascending (partial Fisher-Yates from the identity)."""
    a = list(range(m))
    for i in range(k):
        j = i + rng.next() % (m - i)
        a[i], a[j] = a[j], a[i]
    return sorted(a[:k])


def coverage_size(nocc: int, nvir: int) -> int:
    """|C_min| = C(N_o, 2) C(N_v, 2)."""
    return math.comb(nocc, 2) * math.comb(nvir, 2)


def sample_spaces(eps: np.ndarray, nocc: int, nvir: int, no: int, nv: int, seed: int):
    """Algorithm 1.  Returns (spaces, draws): spaces an int32 array (k, 8) laid out as the
    library's space records (no, nv, occupied orbitals, virtual orbitals as absolute indices,
    unused slots -1), sorted by ascending Delta-eps; draws the number of candidates drawn."""
    if no < 2 or nv < 2 or no > nocc or nv > nvir:
        raise ValueError("active spaces need 2 <= n_o <= N_o and 2 <= n_v <= N_v")
    pair_o = {}
    for a in range(nocc):
        for b in range(a + 1, nocc):
            pair_o[(a, b)] = len(pair_o)
    pair_v = {}
    for a in range(nvir):
        for b in range(a + 1, nvir):
            pair_v[(a, b)] = len(pair_v)
    covered = np.zeros((len(pair_o), len(pair_v)), dtype=bool)
    remaining = covered.size
    rng = SplitMix64(seed)
    kept = []  # (delta_eps, occupied, virtual)
    draws = 0
    while remaining > 0:
        occ = draw(rng, nocc, no)
        vir = draw(rng, nvir, nv)
        draws += 1
        new = []
        for i in range(no):
            for j in range(i + 1, no):
                for a in range(nv):
                    for b in range(a + 1, nv):
                        x, y = pair_o[(occ[i], occ[j])], pair_v[(vir[a], vir[b])]
                        if not covered[x, y]:
                            new.append((x, y))
        if not new:
            continue
        for x, y in new:
            covered[x, y] = True
        remaining -= len(new)
        sv = 0.0
        for a in vir:
            sv = sv + float(eps[nocc + a])
        so = 0.0
        for i in occ:
            so = so + float(eps[i])
        kept.append((sv - so, occ, [nocc + a for a in vir]))
    order = sorted(range(len(kept)), key=lambda t: kept[t][0])  # Python's sort is stable
    out = np.full((len(kept), 8), -1, dtype=np.int32)
    for r, t in enumerate(order):
        _, occ, vir = kept[t]
        out[r, 0], out[r, 1] = no, nv
        out[r, 2:2 + no] = occ
        out[r, 2 + no:2 + no + nv] = vir
    if not covered.all():
        raise AssertionError("the sampled spaces do not cover C_min")
    return out, draws


def covers(spaces: np.ndarray, nocc: int, nvir: int) -> np.ndarray:
    """covered[o1, o2, v1, v2] (o1 < o2, v1 < v2 relative indices) by brute force over the list."""
    cov = np.zeros((nocc, nocc, nvir, nvir), dtype=bool)
    for row in spaces:
        no, nv = int(row[0]), int(row[1])
        occ = [int(x) for x in row[2:2 + no]]
        vir = [int(x) - nocc for x in row[2 + no:2 + no + nv]]
        for i in occ:
            for j in occ:
                for a in vir:
                    for b in vir:
                        if i < j and a < b:
                            cov[i, j, a, b] = True
    return cov
