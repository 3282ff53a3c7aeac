"""The TF32 tcgen05 batched GEMM (building block of the mixed arm's Schur products)
against an FP64 matmul of the same FP32 inputs."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("batch,M,N,K", [(3, 135, 490, 135), (2, 490, 490, 135), (4, 130, 250, 37),
                                         (1, 1, 8, 1), (5, 128, 256, 32), (2, 300, 17, 70)])
def test_tf32_gemm_matches_fp64_reference(batch, M, N, K):
    from paper_1911_02366_gb300 import sc
    g = torch.Generator(device="cuda").manual_seed(batch * 1000 + M + N + K)
    A = torch.randn(batch, M, K, device="cuda", generator=g)
    B = torch.randn(batch, K, N, device="cuda", generator=g)
    C0 = torch.randn(batch, M, N, device="cuda", generator=g)
    C = C0.clone()
    sc.sc_gemm_tf32(A, B, C, alpha=-1.0, beta=1.0, stream=torch.cuda.current_stream().cuda_stream)
    ref = C0.double() - A.double() @ B.double()
    scale = (A.double().abs() @ B.double().abs()).max().item()
    err = (C.double() - ref).abs().max().item() / max(scale, 1e-30)
    # TF32 keeps 10 explicit mantissa bits: per-product error <= 2^-10 relative
    assert err < 2e-3, err
    assert err > 0.0 or K == 1
