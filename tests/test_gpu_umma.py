"""Split-BF16 tensor-core GEMM (tcgen05 + TMA + TMEM) used for the PDEP products of Eq. 3.

C = alpha A B^T + beta C with A, B FP32 split into bf16 hi + lo and three BF16 products.
Two checks per shape: against the same three products computed in FP64 from the same splits
(only FP32 accumulation differs), and against the exact FP64 product within the split-BF16
bound 4 * 2^-18 * (|A| |B|^T).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_20728_gb300 as p
    return p


def _split(x):
    hi = x.to(torch.bfloat16).to(torch.float32)
    lo = (x - hi).to(torch.bfloat16).to(torch.float32)
    return hi.double(), lo.double()


@pytest.mark.parametrize("M,N,K", [(256, 256, 6859), (256, 6859, 256), (1, 1, 1), (130, 7, 65), (300, 129, 1000),
                                   (128, 128, 64)])
def test_bf16x3_gemm(pkg, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 7 * K)
    A = torch.randn(M, K, device="cuda", generator=g)
    B = torch.randn(N, K, device="cuda", generator=g)
    C0 = torch.randn(M, N, device="cuda", generator=g)
    C = C0.clone()
    pkg.bse_gemm_bf16x3(0.5, A, B, -2.0, C)
    Ah, Al = _split(A)
    Bh, Bl = _split(B)
    ref3 = 0.5 * (Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T) - 2.0 * C0.double()
    mag = 0.5 * (A.double().abs() @ B.double().abs().T) + 2.0 * C0.double().abs()
    d3 = (C.double() - ref3).abs()
    assert (d3 <= 4e-6 * mag + 1e-30).all(), d3.max().item()
    exact = 0.5 * A.double() @ B.double().T - 2.0 * C0.double()
    dx = (C.double() - exact).abs()
    assert (dx <= 4 * 2.0 ** -18 * mag + 4e-6 * mag).all(), (dx / mag).max().item()
