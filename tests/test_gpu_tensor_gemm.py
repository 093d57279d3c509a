"""The tcgen05 bf16 GEMM (D = A B^T, fp32 accumulation) against a plain
PyTorch fp32 matmul of the same bf16 operands."""
import pytest

from paper_2311_15429_gb300 import rp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (256, 128, 512), (384, 256, 4096), (1024, 96, 1024),
                                   (128, 224, 192)])
def test_gemm_matches_fp32_reference(M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    rp.rp_gemm_bf16(A, B, D)
    ref = A.float() @ B.float().T
    err = (D - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


def test_gemm_rejects_unsupported_shapes():
    import torch
    A = torch.zeros(100, 64, device="cuda", dtype=torch.bfloat16)
    B = torch.zeros(32, 64, device="cuda", dtype=torch.bfloat16)
    D = torch.zeros(100, 32, device="cuda")
    with pytest.raises(rp.RPError) as e:
        rp.rp_gemm_bf16(A, B, D)
    assert e.value.status == rp.RP_ERR_ARG
