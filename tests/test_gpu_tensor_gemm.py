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


@pytest.mark.parametrize("M,N,K,splits", [(384, 128, 4096, 0), (384, 128, 4096, 7), (128, 64, 640, 10),
                                          (256, 32, 192, 5)])
def test_split_k_matches_fp32_reference(M, N, K, splits):
    """Split-K: chunk sums reduced in a fixed order; some splits may be empty
    (10 chunks of one k-tile each over K = 640, 5 over 3 k-tiles)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(7 * M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda")
    rp.rp_gemm_tn(A, B, D, terms=1, splits=splits)
    ref = A.float() @ B.float().T
    err = (D - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err
    D2 = torch.full((M, N), float("nan"), device="cuda")
    rp.rp_gemm_tn(A, B, D2, terms=1, splits=splits)
    assert torch.equal(D, D2)   # deterministic


@pytest.mark.parametrize("M,N,K,splits", [(384, 128, 2048, 0), (128, 96, 256, 1), (256, 64, 512, 13)])
def test_three_term_split_matches_fp64_product(M, N, K, splits):
    """hi/lo operands: the three-term product reaches about 16-bit operand
    precision, far beyond a single bf16 product of the same fp32 data."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * N + K)
    a = torch.randn(M, K, device="cuda", generator=g)
    b = torch.randn(N, K, device="cuda", generator=g)
    ah = a.to(torch.bfloat16)
    bh = b.to(torch.bfloat16)
    al = (a - ah.float()).to(torch.bfloat16)
    bl = (b - bh.float()).to(torch.bfloat16)
    A = torch.cat([ah, al], 1).contiguous()
    B = torch.cat([bh, bl], 1).contiguous()
    D = torch.full((M, N), float("nan"), device="cuda")
    rp.rp_gemm_tn(A, B, D, terms=3, splits=splits)
    ref = (a.double() @ b.double().T)
    expect = (ah.double() @ bh.double().T + ah.double() @ bl.double().T + al.double() @ bh.double().T)
    scale = ref.abs().max().item()
    assert (D.double() - expect).abs().max().item() / scale < 1e-5
    single = (ah.double() @ bh.double().T - ref).abs().max().item() / scale
    three = (D.double() - ref).abs().max().item() / scale
    assert three < single / 20, (three, single)


@pytest.mark.parametrize("M,N,K,splits", [(256, 320, 256, 1), (128, 64, 2048, 0), (384, 256, 640, 3),
                                          (128, 512, 128, 1)])
def test_fp16_and_column_tiles_match_fp32_reference(M, N, K, splits):
    """fp16 operands; N above 256 runs in column tiles (320 = 2 x 160,
    512 = 2 x 256)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(11 * M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.float16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.float16)
    D = torch.full((M, N), float("nan"), device="cuda")
    rp.rp_gemm_tn(A, B, D, terms=1, splits=splits)
    ref = A.float() @ B.float().T
    err = (D - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err
