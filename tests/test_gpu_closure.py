"""The learned closure's tensor-core kernels against plain references
(GPU).  The GEMM is checked against a float64 numpy product of the same
bf16-rounded operands."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_00304_gb300 as mod
    return mod


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (256, 64, 128), (128, 128, 576), (384, 256, 192),
                                   (256, 32, 64), (640, 48, 576)])
def test_tc_gemm_bf16(lb, M, N, K):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    C0 = torch.randn(M, N, generator=g)
    ref = 0.5 * (A.double().numpy() @ B.double().numpy().T) + 0.25 * C0.double().numpy()
    Ad, Bd, Cd = A.cuda(), B.cuda(), C0.clone().cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    lb.lbmpcd_tc_gemm_bf16(Ad, Bd, Cd, alpha=0.5, beta=0.25, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = Cd.cpu().double().numpy()
    scale = np.abs(A.double().numpy()) @ np.abs(B.double().numpy()).T
    assert np.max(np.abs(got - ref) / (0.5 * scale + 1e-6)) < 1e-5
