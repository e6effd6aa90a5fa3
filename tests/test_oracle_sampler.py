"""Pins of the active-space sampler (Algorithm 1) and parity of the library's host sampler.

The sampler is stochastic, but the size of a cycle concentrates: for the paper's systems the
mean count over seeds must lie within 2 % of the cycle sizes the paper prints
(tests/golden/paper_cycle_sizes.json).  Exact special cases: (2,2) spaces cover one tuple each,
so the cycle is every (2,2) space; an all-orbital space covers everything at once.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import sampler

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_cycle_sizes.json")


def _eps(nocc, nvir, seed=0):
    rng = np.random.default_rng(seed)
    return np.concatenate([np.sort(rng.normal(-1.0, 0.3, nocc)), np.sort(rng.normal(1.0, 0.5, nvir))])


@pytest.mark.parametrize("name", ["h2o_cc-pVDZ", "h2o_aug-cc-pVDZ", "h2o_cc-pVTZ", "h2o_aug-cc-pVTZ",
                                  "h2o_cc-pVQZ", "propane_cc-pVDZ"])
def test_cycle_sizes_match_the_paper(name):
    g = json.load(open(GOLDEN))[name]
    no, nv, paper = g["nocc"], g["nvir"], g["spaces"]
    seeds = range(1, 3) if no > 4 else range(1, 7)
    counts = []
    for s in seeds:
        sp, draws = sampler.sample_spaces(_eps(no, nv), no, nv, 3, 3, s)
        counts.append(len(sp))
        assert math.ceil(sampler.coverage_size(no, nv) / 9) <= len(sp) <= draws
    assert abs(np.mean(counts) - paper) / paper < 0.02, (counts, paper)


@pytest.mark.parametrize("nocc,nvir,no,nv", [(4, 19, 3, 3), (6, 12, 3, 3), (5, 9, 2, 3), (6, 10, 3, 2)])
def test_sampled_cycles_cover_and_are_sorted(nocc, nvir, no, nv):
    eps = _eps(nocc, nvir, 3)
    sp, _ = sampler.sample_spaces(eps, nocc, nvir, no, nv, 11)
    cov = sampler.covers(sp, nocc, nvir)
    for i, j in itertools.combinations(range(nocc), 2):
        for a, b in itertools.combinations(range(nvir), 2):
            assert cov[i, j, a, b]
    de = [sum(eps[v] for v in r[2 + no:2 + no + nv]) - sum(eps[o] for o in r[2:2 + no]) for r in sp]
    assert all(x <= y for x, y in zip(de, de[1:]))
    assert len({tuple(r) for r in sp.tolist()}) == len(sp)   # a repeated candidate adds nothing


def test_minimal_spaces_are_every_22_space():
    nocc, nvir = 4, 7
    sp, _ = sampler.sample_spaces(_eps(nocc, nvir), nocc, nvir, 2, 2, 5)
    assert len(sp) == sampler.coverage_size(nocc, nvir)
    got = {tuple(r[2:6]) for r in sp.tolist()}
    want = {(i, j, nocc + a, nocc + b) for i, j in itertools.combinations(range(nocc), 2)
            for a, b in itertools.combinations(range(nvir), 2)}
    assert got == want


def test_all_orbital_space_is_one_space():
    sp, draws = sampler.sample_spaces(_eps(3, 3), 3, 3, 3, 3, 9)
    assert len(sp) == 1 and draws == 1
    assert sp[0].tolist() == [3, 3, 0, 1, 2, 3, 4, 5]


def test_generator_matches_published_outputs():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.json")))
    rng = sampler.SplitMix64(g["seed"])
    assert [rng.next() for _ in g["outputs"]] == [int(x) for x in g["outputs"]]


def test_draws_are_uniform():
    rng = sampler.SplitMix64(123)
    m, k, n = 9, 3, 27000
    hist = np.zeros(math.comb(m, k))
    index = {c: t for t, c in enumerate(itertools.combinations(range(m), k))}
    for _ in range(n):
        hist[index[tuple(sampler.draw(rng, m, k))]] += 1
    exp = n / len(hist)
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < len(hist) + 5 * math.sqrt(2 * len(hist))   # ~ 4.6 sigma above the mean of chi^2(83)


@pytest.fixture(scope="module")
def qf():
    from paper_2606_04186_gb300 import build, qflow
    if not os.path.exists(qflow.LIB_PATH):
        build.build()
    qflow.lib()
    return qflow


@pytest.mark.parametrize("nocc,nvir,no,nv,seed", [(4, 19, 3, 3, 1), (6, 12, 3, 3, 2), (5, 9, 2, 3, 3),
                                                   (4, 7, 2, 2, 4), (8, 30, 3, 3, 5)])
def test_library_sampler_equals_the_oracle(qf, nocc, nvir, no, nv, seed):
    eps = _eps(nocc, nvir, seed)
    ref, draws_ref = sampler.sample_spaces(eps, nocc, nvir, no, nv, seed)
    got, draws = qf.sample_spaces(eps, nocc, no, nv, seed)
    assert draws == draws_ref
    assert np.array_equal(got, ref)


def test_library_sampler_propane_cycle(qf):
    g = json.load(open(GOLDEN))["propane_cc-pVDZ"]
    counts = [len(qf.sample_spaces(_eps(13, 69), 13, 3, 3, s)[0]) for s in range(1, 9)]
    assert abs(np.mean(counts) - g["spaces"]) / g["spaces"] < 0.01, counts


def test_library_sampler_rejects_bad_sizes(qf):
    with pytest.raises(qf.QFlowError):
        qf.sample_spaces(_eps(4, 7), 4, 1, 2, 0)
    with pytest.raises(qf.QFlowError):
        qf.sample_spaces(_eps(4, 7), 4, 5, 2, 0)


def test_sampled_cycle_flow_reaches_ccsd(n10):
    """A cycle that covers every double reaches the CCSD fixed point (every amplitude is owned)."""
    from oracle import ccsd, flow
    eps, h, g, _ = n10
    fd = ccsd.fock_diagonal(h, g, 3)
    sp, _ = sampler.sample_spaces(fd, 3, 7, 3, 3, 21)
    f = flow.Flow(h, g, 3, sp)
    assert f.uncovered() == 0
    e_cc = ccsd.ccsd(h, g, 3, tol=1e-13)[0]
    f.run(tol_e=1e-10, tol_t=1e-9, max_sweeps=60)
    assert abs(f.e_mean - e_cc) < 1e-9
