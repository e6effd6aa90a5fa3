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
