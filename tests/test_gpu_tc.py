"""The BF16 tensor-core GEMM (tcgen05, TMEM accumulation) against a plain FP32 reference (GPU).

Inputs are rounded to BF16 by the kernel; the reference multiplies the same BF16-rounded values
in FP64, so the only difference is FP32 accumulation order (relative ~1e-6 of sum |a b|)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2510_23993_gb300 as chem

DEV = "cuda:0"


def _bf16(x):
    return x.to(torch.bfloat16).to(torch.float64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    chem.build()


@pytest.mark.parametrize("M,N,K,epi,ksplit,transA,transB", [
    (128, 128, 64, 0, 1, False, False),
    (300, 128, 200, 0, 1, False, False),      # ragged M and K
    (257, 10, 128, 1, 1, False, False),        # N not a multiple of 16, bias
    (1000, 128, 12, 2, 1, False, False),       # bias + GELU, K = 12 (first layer)
    (128, 256, 96, 0, 1, True, False),         # transposed A, N = 256
    (128, 128, 4096, 3, 8, True, True),        # weight gradient: K split over 8 CTAs, atomics
])
def test_tc_gemm(M, N, K, epi, ksplit, transA, transB):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(K, M, generator=g) if transA else torch.randn(M, K, generator=g)
    B = torch.randn(K, N, generator=g) if transB else torch.randn(N, K, generator=g)
    bias = torch.randn(N, generator=g)
    dA, dB, dbias = A.to(DEV), B.to(DEV), bias.to(DEV)
    C = torch.zeros(M, N, device=DEV)
    C2 = torch.zeros(M, N, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    sam, sak = (1, M) if transA else (K, 1)
    sbn, sbk = (1, N) if transB else (K, 1)
    rc = chem.chem_tc_gemm(dA, sam, sak, dB, sbn, sbk, C, N, dbias, C2, M, N, K, epi, ksplit, status)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    Am = (A.T if transA else A).double()
    Bm = (B.T if transB else B).double()
    ref = _bf16(Am) @ _bf16(Bm).T
    scale = (_bf16(Am).abs() @ _bf16(Bm).abs().T)
    if epi in (1, 2):
        ref = ref + bias.double()
    got = C.cpu().double()
    err = ((got - ref).abs() / (scale + 1e-30)).max().item()
    assert err < 2e-6, err
    if epi == 2:
        gelu = 0.5 * ref * (1 + torch.erf(ref / 2 ** 0.5))
        assert (C2.cpu().double() - gelu).abs().max().item() < 1e-4 * (1 + gelu.abs().max().item())
