"""Tensor-core GEMM engine (tcgen05, three-term TF32) vs an FP64 product.

The three-term split keeps each product to about 2^-21 relative (the hi part has 11
significant bits, the lo part rounds the remainder to 11 more, the lo*lo term is dropped):
1e-6 times sum_k |A_mk| |B_nk|.  The tensor cores' FP32 accumulator drops the bits below its
last place at every instruction, so the bound adds one FP32 ulp of the result per K = 8
instruction of the large term: ceil(K / 8) * 2^-23 * |C|.
"""
import numpy as np
import pytest

from gpu_util import library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return library()


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (200, 150, 77), (1, 300, 5), (384, 256, 720), (100, 5184, 100)])
def test_gemm_matches_fp64(qf, M, N, K):
    import torch
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    At, Bt = torch.as_tensor(A, device="cuda"), torch.as_tensor(B, device="cuda")
    C = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    qf.gemm_tf32x3_device(At, Bt, C, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    bound = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    got = C.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    acc_bound = np.ceil(K / 8) * 2.0 ** -23 * np.abs(ref)
    assert (np.abs(got - ref) <= 1e-6 * bound + acc_bound + 1e-30).all(), np.abs(got - ref).max()


def test_gemm_empty_and_args(qf):
    import torch
    A = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
    B = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    C = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    qf.gemm_tf32x3_device(A, B, C, err)
    torch.cuda.synchronize()
    assert err.item() == 0
