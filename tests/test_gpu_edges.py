"""Edge cases through the C ABI: the largest orbital count the library takes (n = 128), an empty
space list, spaces whose Davidson runs out of iterations, and non-finite integrals."""
import numpy as np
import pytest

from oracle import cas, ccsd, flow
from paper_2606_04186_gb300 import synth

from gpu_util import library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_largest_orbital_count_first_sweep(qf, precision):
    """n = 128 (4 occupied, 124 virtual), 4,000 sampled (3,3) spaces: the first sweep (bare
    Hamiltonian) against the oracle's CASCI of 12 sampled spaces."""
    n, no = 128, 4
    _, h, g = synth.make_system(n, no, 5.0, 9)
    sp = synth.sampled_spaces(n, no, 4000, 9)
    fl = qf.Flow(h, g, no, sp, precision=precision)
    de, dt, nf, code = fl.sweep(raise_on_fail=False)
    assert nf == 0
    _, per = fl.energy(per_space=True)
    perm = fl.order()
    fl.close()
    occ_idx = np.arange(no)
    F = h + 2.0 * np.einsum("pqkk->pq", g[:, :, occ_idx][:, :, :, occ_idx]) \
        - np.einsum("pkkq->pq", g[:, occ_idx][:, :, occ_idx])
    e_hf = ccsd.hf_energy(h, g, no)
    te = 1e-8 if precision == "fp64" else 1e-6
    for pos in np.random.default_rng(1).choice(len(sp), 12, replace=False):
        occ, vir = flow.space_orbitals(sp[perm[pos]])
        e_ref = cas.solve_space(e_hf, F, g, occ, vir)[0]
        assert abs(per[pos] - e_ref) < te


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_empty_space_list(qf, precision):
    _, h, g, _ = synth.system_inputs("n10", with_spaces=False)
    sp = np.zeros((0, 8), dtype=np.int32)
    fl = qf.Flow(h, g, 3, sp, precision=precision)
    assert fl.init_status == qf.WARN_UNCOVERED   # no space owns anything
    de, dt, nf, code = fl.sweep()
    assert code == qf.OK and nf == 0 and dt == 0.0
    assert fl.energy() == 0.0
    t1, t2 = fl.amplitudes()
    assert not t1.any() and not t2.any()
    fl.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spaces_out_of_iterations_keep_their_amplitudes(qf, precision):
    """An iteration limit at the median of what n24's first sweep needs: spaces that need more
    report status 1, the sweep returns QFLOW_ERR_NOCONV with their count, and the amplitudes they
    own stay at their old value (zero); converged spaces match the run without the limit."""
    _, h, g, sp = synth.system_inputs("n24")
    s = synth.SYSTEMS["n24"]
    full = qf.Flow(h, g, s.nocc, sp, precision=precision)
    full.sweep()
    it_f, _ = full.stats()
    limit = max(1, int(np.median(it_f)))
    short = qf.Flow(h, g, s.nocc, sp, precision=precision, max_iter=limit)
    de, dt, nf, code = short.sweep(raise_on_fail=False)
    it, st = short.stats()
    assert code == qf.ERR_NOCONV and nf == int((st != 0).sum()) > 0
    assert set(np.unique(st).tolist()) <= {0, 1}
    _, per_s = short.energy(per_space=True)
    _, per_f = full.energy(per_space=True)
    assert np.isfinite(per_s).all()
    ok = st == 0
    assert ok.any()
    assert np.abs(per_s[ok] - per_f[ok]).max() < (1e-12 if precision == "fp64" else 1e-6)
    t1, t2 = short.amplitudes()
    _, o1, o2, _ = qf.plan(h, g, s.nocc, sp)
    failed = set(np.nonzero(st != 0)[0].tolist())
    assert all(t1[i, a] == 0.0 for i, a in zip(*np.nonzero(np.isin(o1, list(failed)))))
    assert all(t2[i, j, a, b] == 0.0 for i, j, a, b in zip(*np.nonzero(np.isin(o2, list(failed)))))
    short.close()
    full.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_non_finite_integrals_are_reported(qf, precision):
    _, h, g, sp = synth.system_inputs("n10")
    h = h.copy()
    h[1, 4] = h[4, 1] = np.nan
    fl = qf.Flow(h, g, 3, sp, precision=precision)
    de, dt, nf, code = fl.sweep(raise_on_fail=False)
    assert code == qf.ERR_NONFINITE
    fl.close()
