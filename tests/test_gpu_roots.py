"""Root selection on the GPU against the oracle, through the C ABI.

* A space whose Phi-dominant root is not its lowest (the first virtual orbital lowered below the
  highest occupied one): both sides take the Phi-dominant root, energies and increments agree.
* A space whose Phi-dominant root is one of a complex pair: the oracle flags it (status 1), the
  GPU reports QFLOW's root status (2), and the amplitudes the space owns keep their value.
"""
import numpy as np
import pytest

from oracle import cas, flow
from paper_2606_04186_gb300 import synth

import planted
from gpu_util import dev, library

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-8, 1e-7), "mixed": (1e-6, 1e-5)}
SPACE_ROOT = 2


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


def _solve(qf, n, no, e0, F, W, k, sps, t1, t2, precision):
    import torch
    own1, own2 = flow.owner_maps(sps, no, n - no)
    ns = len(sps)
    energy = torch.zeros(ns, dtype=torch.float64, device="cuda")
    status = torch.full((ns,), -1, dtype=torch.int32, device="cuda")
    iters = torch.zeros(ns, dtype=torch.int32, device="cuda")
    t1o, t2o = dev(t1), dev(t2)
    t1n, t2n = t1o.clone(), t2o.clone()
    qf.solve_device(n, no, dev(np.array([e0])), dev(F), dev(W), k, dev(sps), energy, status, iters,
                    owner1=dev(own1.astype(np.int32)), owner2=dev(own2.astype(np.int32)), t1_old=t1o, t2_old=t2o,
                    t1_new=t1n, t2_new=t2n, precision=precision)
    torch.cuda.synchronize()
    return (energy.cpu().numpy(), status.cpu().numpy(), iters.cpu().numpy(), t1n.cpu().numpy(), t2n.cpu().numpy(),
            own1, own2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_phi_dominant_root_above_the_lowest(qf, k, precision):
    _, h, g, _ = synth.system_inputs("n10", with_spaces=False)
    n, no = 10, 3
    e0, F, W = planted.lowered_virtual(h, g, no)
    sps = synth.all_spaces(n, no, k, k)
    t1 = np.zeros((no, n - no))
    t2 = np.zeros((no, no, n - no, n - no))
    E, st, it, t1n, t2n, own1, own2 = _solve(qf, n, no, e0, F, W, k, sps, t1, t2, precision)
    ref = flow.solve_all(e0, F, W, sps)
    assert all(r[3] == 0 for r in ref) and (st == 0).all(), st
    not_lowest = sum(not planted.selected_is_lowest(e0, F, W, *flow.space_orbitals(row)) for row in sps)
    assert not_lowest > 0
    te, tt = TOL[precision]
    Er = np.array([r[0] for r in ref])
    assert np.abs(E - Er).max() < te
    t1r, t2r = flow.merge(t1, t2, sps, ref, own1, own2, no)
    assert np.abs(t1n - t1r).max() < tt and np.abs(t2n - t2r).max() < tt


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_complex_phi_dominant_root_is_flagged(qf, k, precision):
    n, no, e0, F, W, sps = planted.complex_pair(k)
    occ, vir = flow.space_orbitals(sps[0])
    assert cas.solve_space(e0, F, W, occ, vir)[3] == 1
    t1 = np.full((no, n - no), 0.125)
    t2 = np.full((no, no, n - no, n - no), -0.25)
    E, st, it, t1n, t2n, own1, own2 = _solve(qf, n, no, e0, F, W, k, sps, t1, t2, precision)
    assert st[0] == SPACE_ROOT, (st, it)
    assert it[0] < 60
    assert np.array_equal(t1n, t1) and np.array_equal(t2n, t2)
