"""Pins of the oracle's root selection and of the merge rule for flagged spaces.

The selected root is the eigenvector with the largest |Phi component|, not the lowest eigenvalue;
a selected root that is complex flags the space (status 1), and a flagged space adds no
increment: the amplitudes it owns keep their value.
"""
import numpy as np
import pytest

from oracle import cas, flow
from paper_2606_04186_gb300 import synth

import planted


@pytest.mark.parametrize("k", [1, 2, 3])
def test_planted_complex_pair_is_flagged(k):
    n, no, e0, F, W, sp = planted.complex_pair(k)
    occ, vir = flow.space_orbitals(sp[0])
    c, h, w = cas.space_problem(e0, F, W, occ, vir)
    mat = cas.cas_matrix(no, n - no, c, h, w)
    ev = np.linalg.eigvals(mat)
    assert np.abs(ev.imag).max() > 1e-3          # the planted pair is there
    e, x1, x2, st = cas.solve_space(e0, F, W, occ, vir)
    assert st == 1
    t1 = np.full((no, n - no), 0.125)
    t2 = np.full((no, no, n - no, n - no), -0.25)
    own1, own2 = flow.owner_maps(sp, no, n - no)
    assert (own1 == 0).all()                     # the one space owns every amplitude
    t1n, t2n = flow.merge(t1, t2, sp, [(e, x1, x2, st)], own1, own2, no)
    assert np.array_equal(t1n, t1) and np.array_equal(t2n, t2)


def test_lowered_virtual_selects_phi_dominant_root_above_the_lowest():
    _, h, g, sp = synth.system_inputs("n10")
    e0, F, W = planted.lowered_virtual(h, g, 3)
    not_lowest = 0
    for row in sp:
        occ, vir = flow.space_orbitals(row)
        e, x1, x2, st = cas.solve_space(e0, F, W, occ, vir)
        assert st == 0
        not_lowest += (not planted.selected_is_lowest(e0, F, W, occ, vir))
    # every space holding orbitals 2 and 3 (15 of the 35) has a lower, doubles-dominated root
    assert not_lowest >= 10
