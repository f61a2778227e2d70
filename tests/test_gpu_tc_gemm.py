"""Tensor-core BF16 GEMM (tcgen05, FP32 accumulation) against a plain PyTorch FP32 product."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2501_17529_b300.csrc import build
    build.build()


# the last two shapes give >= 120 tiles of 128 x 256: the wide-tile kernel
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (512, 256, 3200), (128, 1024, 256),
                                   (4096, 1024, 192), (7680, 512, 3072)])
@pytest.mark.parametrize("epi", ["plain", "bias_relu", "bf16_out"])
def test_gemm_matches_fp32_reference(M, N, K, epi):
    from paper_2501_17529_b300.dcflow import dcflow_gemm_bf16
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g) if epi == "bias_relu" else None
    out = dcflow_gemm_bf16(A, B, bias=bias, relu=(epi == "bias_relu"), out_bf16=(epi == "bf16_out"))
    torch.cuda.synchronize()
    ref = A.float() @ B.float().T
    if bias is not None:
        ref = torch.relu(ref + bias)
    err = (out.float() - ref).abs().max().item()
    scale = ref.abs().max().item() + 1.0
    tol = 1e-2 if epi == "bf16_out" else 1e-4
    assert err <= tol * scale, (err, scale)
