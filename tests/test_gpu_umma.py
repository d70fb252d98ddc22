"""The tcgen05 tile GEMM (BF16 in, FP32 accumulate in TMEM) against a plain
FP32 matmul of the same BF16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_01152_gb300 import build
    build.build()


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (128, 256, 64), (300, 64, 200), (1000, 128, 1024),
                                   (257, 96, 72), (4096, 256, 2304)])
def test_gemm_matches_fp32_reference(M, N, K):
    from paper_2507_01152_gb300.ussim import gemm_bf16_nt
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    gemm_bf16_nt(A, B, C, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.double().cpu() @ B.double().cpu().T
    got = C.double().cpu()
    rel = (got - ref).norm() / ref.norm()
    assert rel < 1e-5, float(rel)
