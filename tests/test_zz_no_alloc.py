"""The allocation-free dressing entry point, called through the C ABI.

It is meant for callers that cannot allocate device memory themselves (memory owned by another
allocator, no implicit synchronisation allowed, fixed budgets).  It must return what the
regular entry point with a caller-provided workspace returns, on two calls in a row (the static
scratch keeps the previous call's contents), and refuse problems larger than its scratch.
"""
import numpy as np
import pytest

from paper_2606_04186_gb300 import synth

from gpu_util import dev, library

pytestmark = pytest.mark.gpu


def _out(n):
    import torch
    return (torch.zeros(1, dtype=torch.float64, device="cuda"),
            torch.zeros((n, n), dtype=torch.float64, device="cuda"),
            torch.zeros((n,) * 4, dtype=torch.float64, device="cuda"))


def test_static_dress_matches_workspace_version_twice():
    import torch
    qf = library()
    eps, h, g, _ = synth.system_inputs("n24", with_spaces=False)
    n, no = 24, 5
    hd, gd = dev(h), dev(g)
    for seed in (3, 4):  # two calls in a row with different pools
        t1, t2 = synth.random_amplitudes(no, n - no, seed, 0.01, 0.02)
        t1d, t2d = dev(t1), dev(t2)
        e0a, Fa, Wa = _out(n)
        work = torch.zeros(qf.dress_workspace(n, no), dtype=torch.uint8, device="cuda")
        qf.dress_device(hd, gd, t1d, t2d, no, e0a, Fa, Wa, work)
        e0b, Fb, Wb = _out(n)
        qf.dress_device_static(hd, gd, t1d, t2d, no, e0b, Fb, Wb)
        torch.cuda.synchronize()
        assert abs(e0a.item() - e0b.item()) < 1e-12
        assert (Fa - Fb).abs().max().item() < 1e-12
        assert (Wa - Wb).abs().max().item() < 1e-12


def test_static_dress_rejects_oversized_problem():
    qf = library()
    n, no = 82, 10
    assert qf.dress_workspace(n, no) > qf.static_scratch_bytes()
    import torch
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(qf.QFlowError) as err:
        qf.dress_device_static(torch.zeros((n, n), dtype=torch.float64, device="cuda"), z, z, z, no, z, z, z)
    assert err.value.code == qf.ERR_TOO_LARGE
