"""The learned closure's tensor-core kernels against plain references
(GPU).  The GEMM is checked against a float64 numpy product of the same
bf16-rounded operands; the network's forward pass and gradients element by
element against the FP64 oracle of oracle/closure.py (tolerances derived in
tests/net_tolerances.py)."""
import numpy as np
import pytest

from tests.net_tolerances import (FWD_RTOL, GRAD_LAYER_L2, GRAD_RTOL, decision_spread, elem_err, oracle_patches,
                                  rel_l2, rms)

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


@pytest.fixture(scope="module")
def problem():
    """Random inputs and targets, parameters of the initial distribution with
    non-zero biases (the head not negligible)."""
    from oracle import closure as C
    rng = np.random.default_rng(11)
    th = C.init_params(2)
    th = th + rng.normal(0, 0.02, size=th.size)
    x = rng.normal(0, 1, size=(3, 16, 16, 24))
    t = rng.normal(0, 1, size=(3, 16, 16, 3))
    return C, th.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64), \
        t.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def realistic(problem):
    """Inputs and moving-average targets of the oracle's own coupled run."""
    C, th, _, _ = problem
    x, t = oracle_patches()
    return C, th, x, t


def _forward(lb, th, x):
    import torch
    net = lb.Net(8)
    net.set_params(th)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.empty(x.shape[0], 16, 16, 3, dtype=torch.float32, device="cuda")
    net.forward(xd, yd)
    net.close()
    return yd.cpu().double().numpy()


@pytest.mark.parametrize("data", ["problem", "realistic"])
def test_net_forward_matches_oracle(lb, data, request):
    """Every output element against the oracle that rounds to bf16 where the
    kernels do (FWD_RTOL of max(|y|, rms)); against the exact FP64 network no
    further than the bf16 definition itself."""
    C, th, x, _ = request.getfixturevalue(data)
    y = _forward(lb, th, x)
    ye, _ = C.forward(th, x, emulate_bf16=True)
    y64, _ = C.forward(th, x)
    e = elem_err(y, ye)
    d_gpu, d_def = rel_l2(y, y64), rel_l2(ye, y64)
    print(f"{data} forward: max element error vs bf16 oracle {e:.2e} (bound {FWD_RTOL:.2e}); "
          f"rel L2 to the exact network: GPU {d_gpu:.2e}, bf16 definition {d_def:.2e}")
    assert e <= FWD_RTOL
    assert d_gpu <= d_def + 1e-3


@pytest.mark.parametrize("data", ["problem", "realistic"])
def test_net_gradient_matches_oracle(lb, data, request):
    """Parameter gradient of the MSE loss, per layer (weights and biases),
    element by element against the oracle's backward with bf16 rounding
    (GRAD_RTOL of max(|g|, rms of the layer's tensor), or twice the oracle's
    own decision spread on this data where that is larger; relative L2 below
    GRAD_LAYER_L2, likewise), and against the exact FP64 backward no further than the
    bf16 definition itself plus 5e-3.  Random targets and the oracle's own
    moving-average targets (realistic)."""
    import torch
    C, th, x, t = request.getfixturevalue(data)
    net = lb.Net(8)
    net.set_params(th)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    L = net.backward(xd, td)
    g = net.get_params(which=1).astype(np.float64)
    net.close()
    Le, ge = C.backward(th, x, t, emulate_bf16=True)
    L64, g64 = C.backward(th, x, t)
    spread = decision_spread(C, th, x, t)
    assert abs(L - Le) < 2e-3 * Le
    o = 0
    for li, (ci, co) in enumerate(C.LAYERS):
        nW = co * 9 * ci
        for name, sl in (("W", slice(o, o + nW)), ("b", slice(o + nW, o + nW + co))):
            if co == 3 and name == "b":
                # the column centring removes the head's bias: its exact gradient
                # is 0, the GPU's is fp32 rounding of sums of centred terms
                assert np.max(np.abs(ge[sl])) < 1e-12
                assert np.max(np.abs(g[sl])) <= 1e-4 * rms(ge[o:o + nW]), g[sl]
                continue
            e = elem_err(g[sl], ge[sl], rms(ge[sl]))
            l2 = rel_l2(g[sl], ge[sl])
            d_gpu, d_def = rel_l2(g[sl], g64[sl]), rel_l2(ge[sl], g64[sl])
            k = 0 if name == "W" else 2
            tol_e = max(GRAD_RTOL, 2.0 * spread[li, k])
            tol_l2 = max(GRAD_LAYER_L2, 2.0 * spread[li, k + 1])
            print(f"{data} grad {ci}->{co} {name}: max element error {e:.2e} (bound {tol_e:.2e}), rel L2 {l2:.2e} "
                  f"(bound {tol_l2:.2e}) vs bf16 oracle; to exact FP64: GPU {d_gpu:.2e}, bf16 definition {d_def:.2e}")
            assert e <= tol_e, (ci, co, name, e)
            assert l2 <= tol_l2, (ci, co, name, l2)
            assert d_gpu <= d_def + 5e-3, (ci, co, name, d_gpu, d_def)
        o += nW + co


def test_net_training_reduces_loss(lb, problem):
    """Adam steps on a fixed batch drive the MSE loss down."""
    import torch
    C, th, x, t = problem
    net = lb.Net(8)
    net.set_params(th)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    losses = [net.train_step(xd, td, 1e-3) for _ in range(60)]
    print(f"training loss {losses[0]:.4f} -> {losses[-1]:.4f}")
    assert losses[-1] < 0.7 * losses[0]
