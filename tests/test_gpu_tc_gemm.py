"""GPU parity of the tcgen05 BF16 GEMM (C = alpha A B^T + beta C) against an
FP32 PyTorch reference on the same BF16-rounded operands, through the C ABI.
Tolerance: FP32 accumulation of K products of BF16 values -> relative 1e-5
per element group (the inputs are exact in BF16; only the summation order
differs)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1706_02145_gb300 import binding as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    B.load()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 128, 64), (256, 128, 128), (130, 70, 72), (1000, 128, 264),
                                   (7, 5, 8), (3000, 60, 136)])
def test_gemm_bf16_matches_fp32_reference(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    Bm = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C0 = torch.randn(M, N, device="cuda", generator=g)
    ref = 0.5 * (A.float() @ Bm.float().T) + 2.0 * C0
    C = C0.clone()
    B.celes_gemm_bf16(A, Bm, C, alpha=0.5, beta=2.0)
    torch.cuda.synchronize()
    err = (C - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * scale * max(1.0, K / 64), (err, scale)


def test_gemm_rejects_unaligned_k():
    A = torch.zeros(16, 12, device="cuda", dtype=torch.bfloat16)
    Bm = torch.zeros(16, 12, device="cuda", dtype=torch.bfloat16)
    C = torch.zeros(16, 16, device="cuda")
    with pytest.raises(B.CelesError) as e:
        B.celes_gemm_bf16(A, Bm, C)
    assert e.value.code == B.CELES_EINVAL
