"""The allocation-free network forward (GPU).

lbmpcd_net_forward_noalloc serves callers that cannot allocate device memory
at the point where they run the closure network: a host code that keeps
nearly all of the GPU's memory in its own pool, or one whose time-step loop
cannot take the device synchronisation a cudaMalloc or cudaFree may cause.
It runs the same kernels in the same order as lbmpcd_net_forward, with its
scratch in one static device array, so its output must equal that of
lbmpcd_net_forward bit for bit on every call; two calls in a row (the larger
batch first) show that nothing left in the shared scratch by one call leaks
into the next.  The output is also checked element by element against the
FP64 oracle of the network (tolerance derived in tests/net_tolerances.py).
This file is collected last, so that a run that stops at the first failure
has run every other test before it."""
import numpy as np
import pytest

from tests.net_tolerances import FWD_RTOL, elem_err

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
    import torch
    from oracle import closure as C
    assert P <= lb.NET_STATIC_MAX_PATCHES
    th = _params(lb, 21 + P)
    rng = np.random.default_rng(100 + P)
    xh = rng.normal(0, 1, size=(P, 16, 16, 24)).astype(np.float32)
    x = torch.tensor(xh, device="cuda")
    net = lb.Net(P)
    net.set_params(th)
    yref = torch.empty(P, 16, 16, 3, dtype=torch.float32, device="cuda")
    net.forward(x, yref)
    ref = yref.cpu().numpy()
    net.close()
    ye, _ = C.forward(th.astype(np.float64), xh.astype(np.float64), emulate_bf16=True)
    thd = torch.tensor(th, device="cuda")
    for call in range(2):
        y = torch.full((P, 16, 16, 3), float("nan"), dtype=torch.float32, device="cuda")
        lb.lbmpcd_net_forward_noalloc(thd, x, y)
        got = y.cpu().numpy()
        assert np.array_equal(got, ref), (call, float(np.max(np.abs(got - ref))))
        e = elem_err(got, ye)
        print(f"P={P} call {call}: equal to lbmpcd_net_forward; max element error vs the oracle {e:.2e}")
        assert e <= FWD_RTOL, (call, e)


def test_noalloc_forward_rejects_too_many_patches(lb):
    import torch
    P = lb.NET_STATIC_MAX_PATCHES + 1
    th = torch.zeros(int(lb.load_library().lbmpcd_net_num_params()), dtype=torch.float32, device="cuda")
    x = torch.zeros(P, 16, 16, 24, dtype=torch.float32, device="cuda")
    y = torch.zeros(P, 16, 16, 3, dtype=torch.float32, device="cuda")
    with pytest.raises(lb.LbmpcdError) as ei:
        lb.lbmpcd_net_forward_noalloc(th, x, y)
    assert ei.value.code == -6   # LBMPCD_ERR_CAPACITY


def test_noalloc_binding_rejects_bad_tensors(lb):
    """The C side sees only addresses, so the binding refuses, before any
    kernel runs, tensors that would be read or written out of bounds."""
    import torch
    n = int(lb.load_library().lbmpcd_net_num_params())
    th = torch.zeros(n, dtype=torch.float32, device="cuda")
    x = torch.zeros(2, 16, 16, 24, dtype=torch.float32, device="cuda")
    y = torch.zeros(2, 16, 16, 3, dtype=torch.float32, device="cuda")
    bad = [(th[:-1], x, y), (th, x, y[:1]), (th, x, torch.zeros(2, 16, 16, 4, device="cuda")),
           (th, x.double(), y), (th, x.transpose(1, 2), y), (th.cpu(), x, y)]
    for t, xx, yy in bad:
        with pytest.raises(ValueError):
            lb.lbmpcd_net_forward_noalloc(t, xx, yy)
