"""Tensor-core (tcgen05) BF16 GEMM against an FP32 matmul of the same bf16 values."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__

    __graft_entry__.build()
    from paper_1310_5541_gb300 import pcsir

    return pcsir


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 256, 448), (1000, 64, 256), (129, 3, 17), (1, 256, 64)])
def test_gemm_bf16_matches_fp32(pc, M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.float() @ B.float().T
    C = pc.gemm_bf16(A.cuda(), B.cuda())
    torch.cuda.synchronize()
    err = (C.cpu() - ref).abs().max().item()
    assert err <= 1e-4 * (1 + ref.abs().max().item()), err


def test_gemm_bf16_transposed_operands_and_accumulate(pc):
    g = torch.Generator().manual_seed(5)
    At = torch.randn(448, 256, generator=g).to(torch.bfloat16)  # A = At.T  (M = 256, K = 448)
    Bt = torch.randn(448, 192, generator=g).to(torch.bfloat16)  # B = Bt.T  (N = 192)
    ref = At.float().T @ Bt.float()
    A = At.cuda().T
    B = Bt.cuda().T
    C = pc.gemm_bf16(A, B)
    C = pc.gemm_bf16(A, B, C, accumulate=True)
    torch.cuda.synchronize()
    err = (C.cpu() - 2 * ref).abs().max().item()
    assert err <= 1e-4 * (1 + 2 * ref.abs().max().item()), err
