"""The C-ABI library loads here (no GPU) and exports every entry point include/qflow.h declares;
its host planner reproduces the oracle's ordering and ownership bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import ccsd, flow
from paper_2606_04186_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qf():
    from paper_2606_04186_gb300 import build, qflow
    if not os.path.exists(qflow.LIB_PATH):
        build.build()
    qflow.lib()
    return qflow


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "qflow.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qflow_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(qf):
    syms = declared_symbols()
    assert len(syms) >= 15
    L = ctypes.CDLL(qf.LIB_PATH)
    for s in syms:
        assert hasattr(L, s), s


def test_strerror_and_defaults(qf):
    assert qf.strerror(0) == "ok"
    o = qf.default_options("mixed")
    assert o.precision == 1 and o.tol == 1e-6 and o.max_iter == 60


@pytest.mark.parametrize("name", ["n10", "n24", "n40"])
def test_plan_matches_oracle(qf, name):
    eps, h, g, sp = synth.system_inputs(name)
    s = synth.SYSTEMS[name]
    perm, o1, o2, unc = qf.plan(h, g, s.nocc, sp)
    fd = ccsd.fock_diagonal(h, g, s.nocc)
    perm_ref = flow.sort_spaces(sp, fd)
    assert np.array_equal(perm, perm_ref)
    r1, r2 = flow.owner_maps(sp[perm_ref], s.nocc, s.n - s.nocc)
    assert np.array_equal(o1, r1) and np.array_equal(o2, r2)
    assert unc == int((r1 < 0).sum() + (r2 < 0).sum())


def test_plan_rejects_bad_spaces(qf):
    eps, h, g, sp = synth.system_inputs("n10")
    bad = sp.copy()
    bad[0, 2] = 5          # an "occupied" index that is virtual
    with pytest.raises(qf.QFlowError):
        qf.plan(h, g, 3, bad)
    bad = sp.copy()
    bad[0, 0] = 2          # (2,3) is not a supported size class
    with pytest.raises(qf.QFlowError):
        qf.plan(h, g, 3, bad)
    empty = sp[:0]
    perm, o1, o2, unc = qf.plan(h, g, 3, empty)
    assert perm.size == 0 and unc == o1.size + o2.size


def test_init_rejects_bad_arguments_before_any_device_work(qf):
    """Argument errors come back as QFLOW_ERR_ARG with no handle, before the library touches a GPU
    (this runs on a machine without one)."""
    import ctypes as C
    eps, h, g, sp = synth.system_inputs("n10")
    L = qf.lib()
    rows = qf._spaces(sp)

    def init(n, nocc, spaces, opt):
        hdl = C.c_void_p()
        code = L.qflow_init(C.byref(hdl), qf._ptr(h), qf._ptr(g), n, nocc, qf._ptr(spaces), len(spaces),
                            C.byref(opt) if opt is not None else None)
        return code, hdl.value

    for n, nocc in ((129, 3), (1, 0), (10, 10), (10, 0)):
        assert init(n, nocc, rows, None) == (qf.ERR_ARG, None), (n, nocc)
    bad = rows.copy()
    bad[0, 2] = 7                       # an occupied slot that names a virtual orbital
    assert init(10, 3, bad, None) == (qf.ERR_ARG, None)
    bad = rows.copy()
    bad[0, 5], bad[0, 6] = bad[0, 6], bad[0, 5]   # virtual orbitals out of ascending order
    assert init(10, 3, bad, None) == (qf.ERR_ARG, None)
    for field, value in (("precision", 5), ("diis", 1), ("diis", -1), ("guess", 9), ("warps", 16), ("chunk", 17),
                         ("ladder_bn", 48), ("ladder_bn", -64)):
        opt = qf.default_options("mixed")
        setattr(opt, field, value)
        assert init(10, 3, rows, opt) == (qf.ERR_ARG, None), field


def test_queries_reject_a_null_handle(qf):
    """Every handle query answers QFLOW_ERR_ARG for a null handle and writes nothing (no GPU)."""
    import ctypes as C
    L = qf.lib()
    i32, f32 = C.c_int32(-7), (C.c_float * 8)()
    assert L.qflow_schedule(None, C.byref(i32), C.byref(i32), C.byref(i32), C.byref(i32), f32, C.byref(i32)) == qf.ERR_ARG
    assert L.qflow_dress_schedule(None, C.byref(i32), f32, C.byref(i32)) == qf.ERR_ARG
    assert i32.value == -7
