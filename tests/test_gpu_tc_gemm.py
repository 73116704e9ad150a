"""GPU check of the bf16 tensor-core GEMM against a plain PyTorch fp32 reference of the same op
(the bf16 operands widened to fp32, fp32 matmul).  Tolerance: fp32 accumulation-order
differences, 2e-5 of the row's absolute mass sum_k |a_k w_k| (+ bf16 output rounding for GELU)."""
import numpy as np
import pytest

from tests.gpu_common import lib

pytestmark = pytest.mark.gpu

SHAPES = [(128, 64, 64), (300, 192, 64), (1000, 256, 128), (517, 512, 128), (2000, 128, 512),
          (64, 384, 128), (4099, 256, 256), (131, 64, 512)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("epi", [0, 1, 2, 4])
def test_tc_gemm_matches_fp32_reference(M, N, K, epi):
    import torch
    P = lib()
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K + epi)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    W = (torch.randn(N, K, device="cuda", generator=g) / np.sqrt(K)).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    ref = A.float() @ W.float().T + bias
    mass = (A.float().abs() @ W.float().abs().T) + bias.abs()
    if epi == 1:
        C = torch.empty(M, N, device="cuda", dtype=torch.bfloat16)
        P.nqs_gemm_bf16(A, W, bias, C, epilogue=1)
        want = torch.nn.functional.gelu(ref, approximate="tanh")
        err = (C.float() - want).abs()
        tol = 2e-5 * mass + 2 ** -7 * want.abs() + 1e-6
    elif epi == 4:
        # compensated GELU: hi in columns [0, N), lo = bf16(g - hi) in [N, 2N)
        C = torch.empty(M, 2 * N, device="cuda", dtype=torch.bfloat16)
        P.nqs_gemm_bf16(A, W, bias, C, epilogue=4)
        want = torch.nn.functional.gelu(ref, approximate="tanh")
        hi, lo = C[:, :N].float(), C[:, N:].float()
        assert torch.equal(hi.to(torch.bfloat16).float(), hi)
        assert bool(((lo.abs() <= 2 ** -8 * hi.abs()) | (hi == 0)).all())
        err = (hi + lo - want).abs()
        tol = 2e-5 * mass + 2 ** -15 * want.abs() + 1e-6
    elif epi == 2:
        C0 = torch.randn(M, N, device="cuda", generator=g)
        C = C0.clone()
        P.nqs_gemm_bf16(A, W, bias, C, epilogue=2)
        err = (C - (C0 + ref)).abs()
        tol = 2e-5 * (mass + C0.abs()) + 1e-6
    else:
        C = torch.empty(M, N, device="cuda")
        P.nqs_gemm_bf16(A, W, bias, C, epilogue=0)
        err = (C - ref).abs()
        tol = 2e-5 * mass + 1e-6
    bad = (err > tol).sum().item()
    assert bad == 0, f"{bad} of {M * N} entries off; max err {err.max().item():.3e}"
