"""The TF32 tcgen05 batched GEMM (building block of the mixed arm's Schur products and
blocked-LU trailing updates) against an FP64 matmul of the same FP32 inputs."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(3, 135, 490, 135), (2, 490, 490, 135), (4, 130, 250, 37), (1, 1, 8, 1), (5, 128, 256, 32),
          (2, 300, 17, 70), (3, 490, 135, 135), (2, 458, 458, 32), (2, 10, 10, 32), (1, 257, 145, 65)]


@pytest.mark.parametrize("trans_a,trans_b", [(False, False), (False, True), (True, False), (True, True)])
@pytest.mark.parametrize("batch,M,N,K", SHAPES)
def test_tf32_gemm_matches_fp64_reference(batch, M, N, K, trans_a, trans_b):
    from paper_1911_02366_gb300 import sc
    g = torch.Generator(device="cuda").manual_seed(batch * 1000 + M + N + K)
    A = torch.randn(batch, M, K, device="cuda", generator=g)
    B = torch.randn(batch, K, N, device="cuda", generator=g)
    C0 = torch.randn(batch, M, N, device="cuda", generator=g)
    C = C0.clone()
    As = A.transpose(1, 2).contiguous() if trans_a else A
    Bs = B.transpose(1, 2).contiguous() if trans_b else B
    sc.sc_gemm_tf32(As, Bs, C, alpha=-1.0, beta=1.0, stream=torch.cuda.current_stream().cuda_stream,
                    trans_a=trans_a, trans_b=trans_b)
    ref = C0.double() - A.double() @ B.double()
    scale = (A.double().abs() @ B.double().abs()).max().item()
    err = (C.double() - ref).abs().max().item() / max(scale, 1e-30)
    # TF32 keeps 10 explicit mantissa bits: per-product error <= 2^-10 relative
    assert err < 2e-3, err
    assert err > 0.0 or K == 1


def test_tf32_gemm_unaligned_views_and_beta_zero():
    """Leading dimensions that are not multiples of 4 take the scalar staging path."""
    from paper_1911_02366_gb300 import sc
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(2, 77, 51, device="cuda", generator=g)
    B = torch.randn(2, 51, 33, device="cuda", generator=g)
    C = torch.full((2, 77, 33), float("nan"), device="cuda")
    sc.sc_gemm_tf32(A, B, C, alpha=2.0, beta=0.0, stream=torch.cuda.current_stream().cuda_stream)
    ref = 2.0 * (A.double() @ B.double())
    scale = 2.0 * (A.double().abs() @ B.double().abs()).max().item()
    assert torch.isfinite(C).all()
    assert (C.double() - ref).abs().max().item() / scale < 2e-3
