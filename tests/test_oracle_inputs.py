"""Pins of the seeded synthetic inputs (closed forms and invariants)."""
import math

import numpy as np

from paper_2606_04186_gb300 import synth


def test_fock_is_diagonal_eps():
    for n, no, xi, seed in [(10, 3, 3.0, 0), (24, 5, 4.0, 1)]:
        eps, h, g = synth.make_system(n, no, xi, seed)
        o = slice(0, no)
        f = h + 2 * np.einsum("pqkk->pq", g[:, :, o, o]) - np.einsum("pkkq->pq", g[:, o, o, :])
        assert np.abs(f - np.diag(eps)).max() < 1e-12
        assert np.all(np.diff(eps[:no]) >= 0) and np.all(np.diff(eps[no:]) >= 0)
        assert eps[:no].min() >= -1.5 and eps[:no].max() <= -0.5
        assert eps[no:].min() >= 0.2 and eps[no:].max() <= 3.0


def test_eri_symmetry_and_psd():
    eps, h, g = synth.make_system(8, 3, 3.0, 7)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1)]:
        assert np.abs(g - g.transpose(perm)).max() < 1e-15
    m = g.reshape(64, 64)
    assert np.linalg.eigvalsh(m).min() > -1e-12


def test_space_lists():
    sp = synth.all_spaces(24, 5)
    assert sp.shape == (math.comb(5, 3) * math.comb(19, 3), 8) == (9690, 8)
    assert len({tuple(r) for r in sp}) == 9690
    mixed = synth.mixed_spaces(40, 6, 2000, 3)
    for k in (1, 2, 3):
        blk = mixed[mixed[:, 0] == k]
        assert blk.shape[0] == 2000 and np.all(blk[:, 1] == k)
        assert np.all(blk[:, 2:2 + k] < 6) and np.all(blk[:, 2 + k:2 + 2 * k] >= 6)
        assert np.all(np.diff(blk[:, 2:2 + k], axis=1) > 0) and np.all(np.diff(blk[:, 2 + k:2 + 2 * k], axis=1) > 0)
    s33 = mixed[mixed[:, 0] == 3]
    assert len({tuple(r) for r in s33}) == 2000
    samp = synth.sampled_spaces(30, 7, 500, 5)
    assert len({tuple(r) for r in samp}) == 500
