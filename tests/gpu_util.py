"""Helpers shared by the GPU tests (building the library once, torch tensors)."""
import os

import numpy as np


def library():
    from paper_2606_04186_gb300 import build, qflow
    if not os.path.exists(qflow.LIB_PATH):
        build.build()
    qflow.lib()
    return qflow


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def vvvv_four_distinct(nv):
    """Mask of the vvvv elements W[a, e, b, f] whose four virtual indices all differ: the mixed
    dressing of a flow leaves their T2 term out ((k, k) spaces with k <= 3 never read them)."""
    ar = np.arange(nv)
    a, e, b, f = np.meshgrid(ar, ar, ar, ar, indexing="ij", sparse=True)
    return (a != e) & (a != b) & (a != f) & (e != b) & (e != f) & (b != f)


def mixed_flow_w(W, Wr, nocc):
    """The flow's mixed-precision W compared with a fully dressed reference Wr: checks that the
    vvvv elements with four distinct virtual indices are the undressed ones (they differ from Wr)
    and returns W with those elements taken from Wr, for element-wise comparison of the rest."""
    v = slice(nocc, W.shape[0])
    four = vvvv_four_distinct(W.shape[0] - nocc)
    Wv, Wvr = W[v, v, v, v], Wr[v, v, v, v]
    assert np.abs(np.where(four, Wv - Wvr, 0.0)).max() > 1e-6  # the restriction is in effect
    out = W.copy()
    out[v, v, v, v] = np.where(four, Wvr, Wv)
    return out
