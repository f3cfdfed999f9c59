"""The learned closure inside the coupled step (feedback = 2) against the
FP64 oracle (GPU).

Sampling (strip fields, 8-frame input, moving-average target) is compared
with the oracle's directly.  In the loop the oracle runs its own network on
its own input (no GPU value enters it): the two sides agree to 1e-12 through
the first evaluation, where the predictions agree element by element within
the network tolerance; the first imposed populations (one LB update later)
agree within the bound that implies; the imposition itself is checked on
every step against Eq. 2 of the GPU's own density and held prediction."""
import numpy as np
import pytest

from tests import inputs

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


def _pair(lb, cfg):
    import oracle as O
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    o = O.OracleSim(cfg["params"])
    o.set_region(*cfg["region"])
    return g, o


def _theta(seed=3):
    from oracle import closure as C
    rng = np.random.default_rng(seed)
    th = C.init_params(seed) + rng.normal(0, 0.01, size=C.n_params())
    return th.astype(np.float32)


@pytest.mark.parametrize("steps", [20, 70])
def test_sampling_matches_oracle(lb, steps):
    """Without parameters feedback = 2 samples only: the input frames (binary32
    ring) and the moving-average target (binary64) match the oracle; 70 steps
    cover one captured 64-step chunk with its particle sort."""
    cfg = inputs.small_2d(feedback=2)
    g, o = _pair(lb, cfg)
    g.step(steps)
    o.step(steps)
    xg, xo = g.get("CLOSURE_IN"), o.get("CLOSURE_IN")
    assert xg.shape == xo.shape
    assert np.max(np.abs(xg - xo)) < 1e-6 * max(1.0, np.max(np.abs(xo)))
    tg, to = g.get("CLOSURE_TARGET"), o.get("CLOSURE_TARGET")
    assert np.max(np.abs(tg - to)) < 1e-12
    assert np.max(np.abs(g.get("POPS") - o.get("POPS"))) < 1e-12
    g.close()


def _imposed(y, rho, sig, cfg):
    """f_eq(rho_LB, u_bar) (Eq. 2) on the inner-buffer nodes from a network
    output y [P][16][16][3], as the header states the imposition: u_bar =
    sqrt(kT/m) times the mean predicted velocity over the node's r x r fine
    cells (u_x mirrored on the right side), fine row R read from patch
    min(R / 16, ceil(Hy / 16) - 1), whose first row is 16 py (Hy - 16 for the
    last patch); patches side-major.  Returns {(x, y): populations}."""
    import oracle as O
    p = cfg["params"]
    r, ny = p["refine"], p["ny"]
    x0, x1 = cfg["region"]
    cw = p["coupling_width"]
    n_out, n_in = (cw + 1) // 2, cw // 2
    hy = (ny - 2) * r
    npy = -(-hy // 16)
    out = {}
    for side in range(2):
        for col in range(n_in):
            x = x0 + n_out + col if side == 0 else x1 - 1 - n_out - col
            for yn in range(1, ny - 1):
                su = np.zeros(2)
                for a in range(r):
                    for b in range(r):
                        row, xi = (yn - 1) * r + a, (n_out + col) * r + b
                        py = min(row // 16, npy - 1)
                        row0 = hy - 16 if py == npy - 1 else 16 * py
                        su += y[side * npy + py, row - row0, xi, 1:3]
                u = np.array([(-1.0 if side else 1.0) * sig * su[0], sig * su[1], 0.0]) / (r * r)
                out[(x, yn)] = O.feq(9, rho[yn, x], u)
    return out


@pytest.mark.parametrize("interval,before", [(1, 0), (3, 0), (4, 10)])
def test_in_loop_imposition_matches_oracle(lb, interval, before):
    """FP64, steps one at a time, parameters loaded after `before`
    sampling-only steps: the network runs on steps n0, n0 + K, ... with
    n0 = max(7, before), and the LB updates from n0 + 1 on impose the latest
    prediction.  The oracle runs its own network in the loop
    (step_with_closure); no GPU value enters it.  Through step n0 the two
    sides agree to 1e-12; the GPU's prediction at n0 matches the oracle's
    element by element (FWD_RTOL); at n0 + 1 the imposed populations differ by
    at most 1.5 rho |delta u_bar|, |delta u_bar| bounded by that tolerance, and
    no other node differs.  On every step from n0 + 1 the GPU's inner-buffer
    populations are f_eq of its own LB density and the prediction held after
    the step before (1e-12), and predictions are held between evaluations."""
    from tests.net_tolerances import FWD_RTOL, elem_err, rms
    cfg = inputs.small_2d(feedback=2)
    p = cfg["params"]
    ny, nx = p["ny"], p["nx"]
    sig = np.sqrt(p["kT"] / p["mass"])
    th = _theta()
    g, o = _pair(lb, cfg)
    g.step(before)
    o.step(before)
    g.set_closure(th, interval=interval)
    o.set_closure(th.astype(np.float64), interval=interval)
    first = max(7, before)
    y_held = None
    for n in range(before, first + 3 * interval + 2):
        g.step(1)
        o.step_with_closure(1)
        fg = g.get("POPS").reshape(9, ny, nx)
        if n <= first:
            xo = o.get("CLOSURE_IN")
            assert np.max(np.abs(g.get("CLOSURE_IN") - xo)) < 1e-6 * max(1.0, np.max(np.abs(xo)))
            assert np.max(np.abs(fg - o.get("POPS").reshape(9, ny, nx))) < 1e-12, n
        if n < first:
            continue
        if n > first:   # imposed by this step's LB update: the prediction held after step n - 1
            imp = _imposed(y_held, g.get("RHO").reshape(ny, nx), sig, cfg)
            for (x, y), want in imp.items():
                assert np.max(np.abs(fg[:, y, x] - want)) < 1e-12 * max(1.0, np.max(np.abs(want))), (n, x, y)
        if n == first + 1:
            yo = o._cl_y
            du = sig * FWD_RTOL * max(float(np.max(np.abs(yo))), rms(yo))
            fo = o.get("POPS").reshape(9, ny, nx)
            mask = np.ones((ny, nx), bool)
            for (x, y) in imp:
                mask[y, x] = False
                assert np.max(np.abs(fg[:, y, x] - fo[:, y, x])) <= 1.5 * fo[:, y, x].sum() * du, (x, y)
            assert np.max(np.abs(fg[:, mask] - fo[:, mask])) < 1e-12
        yg = g.get("CLOSURE_OUT").reshape(-1, 16, 16, 3)
        if (n - first) % interval:
            np.testing.assert_array_equal(yg, y_held)      # held between evaluations
        if n == first:
            assert elem_err(yg, o._cl_y) <= FWD_RTOL
        y_held = yg
    # the imposition did change the inner columns relative to one-way coupling
    one = lb.Lbmpcd(cfg["params"])
    one.set_region(0, *cfg["region"])
    one.step(n + 1)
    assert np.max(np.abs(one.get("POPS") - g.get("POPS"))) > 1e-6
    g.close()
    one.close()


def test_in_loop_closure_fp32_graph(lb):
    """FP32 with the closure evaluated every 8 steps in captured graphs (a
    64-step chunk and the powers of two below it, the network node enabled on
    the evaluation steps only): the run stays finite, the last evaluation
    (step 127) is the network of that step's input (checked through the
    allocation-free forward, which the allocation-free tests tie to the
    oracle), and the populations the LB update of step 127 imposed are f_eq of
    the LB density and the prediction held before it."""
    import torch
    cfg = inputs.small_2d(feedback=2, precision=1)
    p = cfg["params"]
    ny, nx = p["ny"], p["nx"]
    th = _theta(5)
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    g.set_closure(th, interval=8)
    g.step(127)
    y_held = g.get("CLOSURE_OUT").reshape(-1, 16, 16, 3)   # imposed by the LB update of step 127
    g.step(1)
    xg = g.get("CLOSURE_IN").reshape(-1, 16, 16, 24)
    yg = g.get("CLOSURE_OUT").reshape(-1, 16, 16, 3)
    P = xg.shape[0]
    y2 = torch.empty(P, 16, 16, 3, dtype=torch.float32, device="cuda")
    lb.lbmpcd_net_forward_noalloc(torch.tensor(th, device="cuda"),
                                  torch.tensor(xg.astype(np.float32), device="cuda"), y2)
    from tests.net_tolerances import FWD_RTOL, elem_err
    # two tensor-core paths (the fused in-loop kernel and the GEMM forward), each
    # within FWD_RTOL of the bf16 network
    assert elem_err(yg, y2.cpu().double().numpy()) <= 2 * FWD_RTOL
    fg = g.get("POPS").reshape(9, ny, nx)
    imp = _imposed(y_held, g.get("RHO").reshape(ny, nx), np.sqrt(p["kT"] / p["mass"]), cfg)
    for (x, y), want in imp.items():
        assert np.max(np.abs(fg[:, y, x] - want)) < 1e-6 * max(1.0, np.max(np.abs(want))), (x, y)
    assert np.all(np.isfinite(g.get("POPS")))
    assert np.all(np.isfinite(g.get("PART_VEL")))
    # unloading the parameters leaves sampling only
    g.set_closure(None)
    g.step(3)
    g.close()


def test_closure_argument_errors(lb):
    cfg = inputs.small_2d(feedback=1)
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    with pytest.raises(lb.LbmpcdError) as ei:
        g.set_closure(_theta())
    assert ei.value.code == -5                        # STATE: no closure replica
    g.close()
    cfg = inputs.small_2d(feedback=2)
    g = lb.Lbmpcd(cfg["params"])
    with pytest.raises(lb.LbmpcdError) as ei:
        g.set_region(0, 20, 34)                       # 28 fine columns < 32
    assert ei.value.code == -1
    g.set_region(0, *cfg["region"])
    with pytest.raises(lb.LbmpcdError) as ei:
        g.set_closure(np.zeros(10, np.float32))
    assert ei.value.code == -1
    g.close()
    with pytest.raises(lb.LbmpcdError):
        lb.Lbmpcd(inputs.small_3d(feedback=2)["params"])
