"""The tcgen05 BF16 GEMM (FP32 accumulation) against float64 matmuls of the same
bf16 values: ragged M and N (N up to several 256-wide tiles), K from one stage to
many trips around the stage ring, every epilogue mode, split-K."""
import ctypes

import numpy as np
import pytest

from paper_2602_22625_gb300 import dbmp as D
from _helpers import cuda, torch

pytestmark = pytest.mark.gpu


def gemm(A, B, mode, bias=None, split_k=1, out=None):
    L = D.load()
    L.dbmp_gemm_bf16.restype = ctypes.c_int32
    L.dbmp_gemm_bf16.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                 ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    M, K = A.shape
    N = B.shape[0]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    if mode == 2:
        C = torch.zeros(M, N, dtype=torch.bfloat16, device="cuda")
        cf, cb = None, C.data_ptr()
    else:
        C = out if out is not None else torch.zeros(M, N, dtype=torch.float32, device="cuda")
        cf, cb = C.data_ptr(), None
    D._check(L.dbmp_gemm_bf16(A.data_ptr(), K, B.data_ptr(), K, M, N, K, mode, cf, cb, N,
                              None if bias is None else bias.data_ptr(), split_k, status.data_ptr(),
                              torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert status.item() == 0
    return C


def operands(M, N, K, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    ref = A.double() @ B.double().T
    return A, B, ref


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 32, 64), (300, 70, 192), (1000, 256, 512),
                                   (77, 5, 128), (4096, 64, 2048), (512, 600, 1024), (256, 1024, 4096)])
def test_gemm_store_f32(M, N, K):
    cuda()
    A, B, ref = operands(M, N, K, M + N + K)
    C = gemm(A, B, 0)
    err = (C.double() - ref).abs().max().item()
    assert err <= 2e-6 * K * 4, err   # fp32 accumulation of K products of size ~1


def test_gemm_split_k_atomic():
    cuda()
    A, B, ref = operands(200, 96, 1024, 5)
    C = gemm(A, B, 1, split_k=4)
    assert (C.double() - ref).abs().max().item() <= 1e-2


def test_gemm_bias_modes():
    cuda()
    A, B, ref = operands(257, 48, 256, 6)
    bias = torch.randn(48, device="cuda")
    C2 = gemm(A, B, 2, bias=bias)
    want = torch.relu(ref + bias.double())
    assert (C2.double() - want).abs().max().item() <= 0.01 * want.abs().max().item() + 1e-3
    assert torch.all(C2.float() >= 0)
    C3 = gemm(A, B, 3, bias=bias)
    assert (C3.double() - (ref + bias.double())).abs().max().item() <= 2e-3


def gemm_mn(A, B, M, N, K, mode, a_mn, b_mn, lda, ldb, split_k=1):
    """A, B given as stored (K-major: M x K / N x K; MN-major: K x M / K x N)."""
    L = D.load()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    flags = (16 if a_mn else 0) | (32 if b_mn else 0)
    D._check(L.dbmp_gemm_bf16(A.data_ptr(), lda, B.data_ptr(), ldb, M, N, K, mode | flags, C.data_ptr(), None,
                              N, None, split_k, status.data_ptr(), torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert status.item() == 0
    return C


@pytest.mark.parametrize("a_mn,b_mn", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", [(128, 256, 128), (300, 200, 320), (64, 512, 1024), (32, 128, 4096)])
def test_gemm_mn_major_operands(M, N, K, a_mn, b_mn):
    """Operands given MN-major (A as K x M, B as K x N, M / N contiguous), as the
    proposal network's weight and input gradients read them."""
    cuda()
    A, B, ref = operands(M, N, K, 7 * M + N + K)
    At = A.T.contiguous() if a_mn else A
    Bt = B.T.contiguous() if b_mn else B
    lda = M if a_mn else K
    ldb = N if b_mn else K
    if (a_mn and lda % 8) or (b_mn and ldb % 8):
        pytest.skip("row stride must be a multiple of 8")
    C = gemm_mn(At, Bt, M, N, K, 0, a_mn, b_mn, lda, ldb)
    err = (C.double() - ref).abs().max().item()
    assert err <= 2e-6 * K * 4, err
    if K >= 1024:   # split-K with atomics on the same layouts
        C1 = gemm_mn(At, Bt, M, N, K, 1, a_mn, b_mn, lda, ldb, split_k=4)
        assert (C1.double() - ref).abs().max().item() <= 2e-6 * K * 4


def test_gemm_wait_timeout_sets_status_and_leaves_the_context_usable():
    """Failure detection without a fault: with the test flag the producer issues no
    copies, the pipeline's bounded waits run out after 2 s, the kernel returns and the
    status word reads DBMP_ERR_TIMEOUT; C is not written and the next GEMM runs."""
    cuda()
    L = D.load()
    A, B, ref = operands(256, 128, 128, 7)
    C = torch.full((256, 128), -7.0, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gemm(A, B, 0)   # declares the argument types
    D._check(L.dbmp_gemm_bf16(A.data_ptr(), 128, B.data_ptr(), 128, 256, 128, 128, 0 | 64, C.data_ptr(), None,
                              128, None, 1, status.data_ptr(), torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert status.item() == D.DBMP_ERR_TIMEOUT
    assert bool((C == -7.0).all())
    C2 = gemm(A, B, 0)
    assert (C2.double() - ref).abs().max().item() <= 2e-6 * 128 * 4
