"""CPU check of the scratch-address cache of the allocation-free dressing entry point.

The entry point keeps the device address of its static scratch array per device and context;
a re-created context (a device reset) must trigger a new look-up instead of reusing an address
that is no longer mapped.  The cache is plain host C++; this compiles a small program around it
with the host compiler and runs it.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_cache_is_keyed_on_device_and_context(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "scratch_cache_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", os.path.join(HERE, "native", "scratch_cache_check.cpp"),
                    "-o", exe], check=True)
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == "ok"
