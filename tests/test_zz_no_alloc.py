"""The allocation-free dressing entry point, called through the C ABI.

It is meant for callers that cannot allocate device memory themselves (memory owned by another
allocator, no implicit synchronisation allowed, fixed budgets).  It must return what the
regular entry point with a caller-provided workspace returns, on two calls in a row (the static
scratch keeps the previous call's contents), leave the device's free memory unchanged, accept
the largest size its header promises (40 orbitals, 6 occupied), refuse problems larger than its
scratch, and refuse to do its first address look-up while the stream is being captured.
"""
import os
import subprocess
import sys

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


@pytest.mark.parametrize("name,n,no", [("n24", 24, 5), ("n40", 40, 6)])
def test_static_dress_matches_workspace_version_twice(name, n, no):
    import torch
    qf = library()
    assert qf.dress_workspace(n, no) <= qf.static_scratch_bytes()
    eps, h, g, _ = synth.system_inputs(name, with_spaces=False)
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


def test_static_dress_allocates_nothing():
    import torch
    qf = library()
    eps, h, g, _ = synth.system_inputs("n24", with_spaces=False)
    n, no = 24, 5
    hd, gd = dev(h), dev(g)
    t1, t2 = synth.random_amplitudes(no, n - no, 5, 0.01, 0.02)
    t1d, t2d = dev(t1), dev(t2)
    e0, F, W = _out(n)
    qf.dress_device_static(hd, gd, t1d, t2d, no, e0, F, W)  # warm-up: kernels loaded, address set up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        qf.dress_device_static(hd, gd, t1d, t2d, no, e0, F, W)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


_CAPTURE_SCRIPT = r"""
import sys
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[2])
import torch
from gpu_util import library
qf = library()
n, no = 10, 3
z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
h, g, t1, t2 = z(n, n), z(n, n, n, n), z(no, n - no), z(no, no, n - no, n - no)
e0, F, W = z(1), z(n, n), z(n, n, n, n)
torch.cuda.synchronize()
s = torch.cuda.Stream()
graph = torch.cuda.CUDAGraph()
code = 0
with torch.cuda.graph(graph, stream=s):
    try:
        qf.dress_device_static(h, g, t1, t2, no, e0, F, W, stream=s.cuda_stream)
    except qf.QFlowError as err:
        code = err.code
print("code", code, qf.ERR_STATE)
"""


def test_first_call_under_capture_is_refused():
    # A fresh process, so that its first call is the one made while the stream is captured.
    here = os.path.dirname(os.path.abspath(__file__))
    res = subprocess.run([sys.executable, "-c", _CAPTURE_SCRIPT, os.path.dirname(here), here],
                         capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    line = [x for x in res.stdout.splitlines() if x.startswith("code")][-1].split()
    assert int(line[1]) == int(line[2])
