"""The tensor-core BF16 GEMM (tcgen05, FP32 accumulation in TMEM) against an FP64 matmul of
the same BF16 values. FP32 accumulation of K products of BF16 values: |error| <= K * 2^-23 *
sum |a b| bounds it; the test uses 2^-18 of the summed magnitudes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1811_00156_gb300 import aiwcrf
    return aiwcrf


def _check(A, M, N, K, at=False, bt=False, ksplit=1, seed=0):
    g = torch.Generator().manual_seed(seed)
    a = torch.randn((K, M) if at else (M, K), generator=g).to(torch.bfloat16)
    b = torch.randn((K, N) if bt else (N, K), generator=g).to(torch.bfloat16)
    c = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    A.aiwcrf_tc_gemm_bf16(a.cuda(), b.cuda(), c, a_trans=at, b_trans=bt, ksplit=ksplit)
    torch.cuda.synchronize()
    a64 = (a.T if at else a).double()
    b64 = (b.T if bt else b).double()
    ref = a64 @ b64.T
    bound = (a64.abs() @ b64.abs().T) * 2.0 ** -18 + 1e-30
    err = (c.double().cpu() - ref).abs()
    assert torch.isfinite(c).all()
    assert (err <= bound).all(), float((err / bound).max())


def test_tc_gemm_single_tile(A):
    _check(A, 128, 64, 64)


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (256, 256, 256), (300, 16, 56), (4096, 256, 64), (129, 32, 520)])
def test_tc_gemm_shapes(A, M, N, K):
    _check(A, M, N, K, seed=M + N + K)


@pytest.mark.parametrize("at,bt", [(False, True), (True, False), (True, True)])
def test_tc_gemm_transposed_operands(A, at, bt):
    _check(A, 256, 128, 512, at=at, bt=bt, seed=3)


def test_tc_gemm_split_k(A):
    _check(A, 256, 256, 4096, at=True, bt=True, ksplit=16, seed=4)
