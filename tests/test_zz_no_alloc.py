"""The allocation-free network forward against the allocating one (GPU).

lbmpcd_net_forward_noalloc runs the same kernels as lbmpcd_net_forward with
its scratch in a static device array; two calls in a row must each match the
handle-based forward, so that nothing left in the scratch by one call leaks
into the next."""
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


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _params(lb, seed):
    """He-normal weights and small random biases, flat in the library's layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (ci, co) in enumerate([(24, 64), (64, 64), (64, 64), (64, 3)]):
        std = np.sqrt(2.0 / (9 * ci)) * (0.1 if li == 3 else 1.0)
        parts.append(rng.normal(0.0, std, size=co * 9 * ci))
        parts.append(rng.normal(0.0, 0.02, size=co))
    th = np.concatenate(parts).astype(np.float32)
    n = int(lb.load_library().lbmpcd_net_num_params())
    assert th.size == n
    return th


@pytest.mark.parametrize("P", [8, 3])
def test_noalloc_forward_matches_net_forward_twice(lb, P):
    """Within the forward tolerance of the closure tests (relative L2 2e-3);
    the two paths run the same kernels in the same order, so they are
    expected to agree bit for bit."""
    import torch
    assert P <= lb.NET_STATIC_MAX_PATCHES
    th = _params(lb, 21 + P)
    rng = np.random.default_rng(100 + P)
    x = torch.tensor(rng.normal(0, 1, size=(P, 16, 16, 24)).astype(np.float32), device="cuda")
    net = lb.Net(P)
    net.set_params(th)
    yref = torch.empty(P, 16, 16, 3, dtype=torch.float32, device="cuda")
    net.forward(x, yref)
    ref = yref.cpu().numpy()
    thd = torch.tensor(th, device="cuda")
    for call in range(2):
        y = torch.full((P, 16, 16, 3), float("nan"), dtype=torch.float32, device="cuda")
        lb.lbmpcd_net_forward_noalloc(thd, x, y)
        got = y.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        e = _rel(got, ref)
        print(f"P={P} call {call}: rel L2 vs lbmpcd_net_forward {e:.2e}, max |diff| {np.max(np.abs(got - ref)):.2e}")
        assert e < 2e-3, (call, e)
    net.close()


def test_noalloc_forward_rejects_too_many_patches(lb):
    import torch
    P = lb.NET_STATIC_MAX_PATCHES + 1
    th = torch.zeros(int(lb.load_library().lbmpcd_net_num_params()), dtype=torch.float32, device="cuda")
    x = torch.zeros(P, 16, 16, 24, dtype=torch.float32, device="cuda")
    y = torch.zeros(P, 16, 16, 3, dtype=torch.float32, device="cuda")
    with pytest.raises(lb.LbmpcdError) as ei:
        lb.lbmpcd_net_forward_noalloc(th, x, y)
    assert ei.value.code == -6   # LBMPCD_ERR_CAPACITY
