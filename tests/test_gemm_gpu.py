"""The tcgen05 BF16 GEMM against an FP64 product of the same BF16 inputs.

Bound: the FP32 accumulator adds K products, so |C - C_ref| <= K 2^-24 sum_k |a_ik b_jk|
(plus the exact BF16 products); the test allows 2 K 2^-24 of that sum.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0908_0681_gb300 import kt  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (128, 256, 64), (256, 256, 352), (200, 48, 64), (1024, 256, 256),
                                   (256, 352, 4096), (384, 96, 80), (1024, 256, 368), (4096, 256, 368),
                                   (8192, 256, 256), (1000, 144, 368)])
def test_gemm_bf16_matches_fp64(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    kt.kt_gemm_bf16(A, B, C, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    a, b = A.double().cpu().numpy(), B.double().cpu().numpy()
    ref = a @ b.T
    bound = 2 * K * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    got = C.double().cpu().numpy()
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= bound).all(), float(np.max(np.abs(got - ref) / bound))


def test_gemm_bf16_rejects_bad_shapes():
    A = torch.zeros((128, 24), dtype=torch.bfloat16, device="cuda")
    B = torch.zeros((16, 24), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((128, 16), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(kt.KtError):
        kt.kt_gemm_bf16(A, B, C, err)      # K = 24 is not a multiple of 16
