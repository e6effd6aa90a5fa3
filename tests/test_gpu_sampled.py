"""Flows over Algorithm 1 cycles on the GPU: parity with the oracle over a sampled n24 cycle and
convergence to CCSD (a cycle covers every double, so every amplitude has an owner)."""
import numpy as np
import pytest

from oracle import ccsd, flow
from paper_2606_04186_gb300 import synth

from gpu_util import library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


@pytest.fixture(scope="module")
def cycle(qf):
    _, h, g, _ = synth.system_inputs("n24", with_spaces=False)
    s = synth.SYSTEMS["n24"]
    sp, _ = qf.sample_spaces(ccsd.fock_diagonal(h, g, s.nocc), s.nocc, 3, 3, 7)
    return h, g, s.nocc, sp


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sampled_cycle_sweeps_match_oracle(qf, cycle, precision):
    h, g, no, sp = cycle
    ref = flow.Flow(h, g, no, sp)
    gpu = qf.Flow(h, g, no, sp, precision=precision)
    assert ref.uncovered() == 0
    te, tt = (1e-8, 1e-7) if precision == "fp64" else (1e-6, 1e-5)
    for _ in range(2):
        ref.sweep()
        gpu.sweep()
        _, per = gpu.energy(per_space=True)
        t1, t2 = gpu.amplitudes()
        assert np.abs(per - ref.energies).max() < te
        assert np.abs(t1 - ref.t1).max() < tt and np.abs(t2 - ref.t2).max() < tt
    gpu.close()


def test_sampled_cycle_converges_to_ccsd(qf, cycle):
    h, g, no, sp = cycle
    e_cc = ccsd.ccsd(h, g, no, tol=1e-12)[0]
    gpu = qf.Flow(h, g, no, sp, precision="fp64")
    for _ in range(60):
        de, dt, nf, code = gpu.sweep()
        if abs(de) < 1e-10 and dt < 1e-9:
            break
    assert abs(gpu.energy() - e_cc) < 1e-8
    gpu.close()
