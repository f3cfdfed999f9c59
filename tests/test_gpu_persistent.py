"""The persistent launch form (one cooperative kernel per chunk, grid barriers
between the LB phase, which also builds the previous step's collision-cell
table, and the particle phase) and the autotuner, against the FP64 oracle
(GPU).  Tolerances as in test_gpu_parity: 1e-12 relative in FP64,
integer results bit-exact."""
import numpy as np
import pytest

import oracle as O
from tests import inputs
from tests.test_gpu_parity import FLOOR, rel_err

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


def _check(g, o):
    assert np.array_equal(g.get("SHIFT"), o.get("SHIFT"))
    assert np.array_equal(g.get("PART_HOME"), o.get("PART_HOME"))
    assert np.array_equal(g.get("PART_CELL"), o.get("PART_CELL"))
    assert np.array_equal(g.get("CELL_COUNT"), o.get("CELL_COUNT"))
    for f in ("PART_POS", "PART_VEL", "CELL_VCM", "WINDOW_MEAN", "POPS", "U"):
        e = rel_err(g.get(f), o.get(f), FLOOR.get(f, 0.0))
        assert e <= 1e-12, (f, e)


@pytest.mark.parametrize("case,bps", [("2d", 0), ("2d", 1), ("3d", 0), ("2d_strip", 0), ("3d_strip", 0)])
def test_persistent_matches_oracle(lb, case, bps):
    """70 steps = chunks of 64, 4 and 2 steps (the particle sort runs before
    the 4-step chunk), then 3 more single steps; also with a near-wall strip
    as the MPCD region."""
    cfg = inputs.small_2d(precision=0, nx=72) if case.startswith("2d") else inputs.small_3d(precision=0, nx=24)
    g = lb.Lbmpcd(cfg["params"])
    o = O.OracleSim(cfg["params"])
    if case.endswith("strip"):
        y1 = 8 if case.startswith("2d") else 6
        g.set_strip(0, y1)
        o.set_strip(y1)
    else:
        g.set_region(0, *cfg["region"])
        o.set_region(*cfg["region"])
    g.set_launch_mode(1, bps)
    g.step(70)
    o.step(70)
    _check(g, o)
    for _ in range(3):
        g.step(1)
        o.step(1)
    _check(g, o)
    g.close()


def test_persistent_uneven_replicas(lb):
    """Three uneven replicas (one without a region) in one persistent launch."""
    reps = [inputs.small_2d(precision=0, seed=31, nx=72),
            inputs.small_2d(precision=0, seed=32, nx=40, ny=14, refine=1, ppc=5),
            inputs.small_2d(precision=0, seed=33, nx=36, ny=20)]
    g = lb.Lbmpcd([r["params"] for r in reps])
    g.set_region(0, *reps[0]["region"])
    g.set_region(1, 10, 30)
    g.set_launch_mode(1)
    o = [O.OracleSim(r["params"], replica=k) for k, r in enumerate(reps)]
    o[0].set_region(*reps[0]["region"])
    o[1].set_region(10, 30)
    g.step(66)
    for k in range(3):
        o[k].step(66)
        e = rel_err(g.get("POPS", k), o[k].get("POPS"))
        assert e <= 1e-12, (k, e)
    for k in (0, 1):
        assert np.array_equal(g.get("PART_HOME", k), o[k].get("PART_HOME"))
        assert rel_err(g.get("PART_VEL", k), o[k].get("PART_VEL")) <= 1e-12
    g.close()


def test_autotune_keeps_the_state_and_the_results(lb):
    """The autotuner times its candidates on a copy: afterwards the handle
    still starts from step 0 and matches the oracle in whatever form it chose."""
    cfg = inputs.small_2d(precision=0, nx=72)
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    choice = g.autotune(steps=64)
    print("autotune choice", choice)
    assert choice["mode"] in (0, 1) and choice["candidates"] >= 3
    o = O.OracleSim(cfg["params"])
    o.set_region(*cfg["region"])
    g.step(67)
    o.step(67)
    _check(g, o)
    g.close()


def test_persistent_mode_rejects_the_closure(lb):
    cfg = inputs.small_2d(feedback=2)
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    with pytest.raises(lb.LbmpcdError) as ei:
        g.set_launch_mode(1)
    assert ei.value.code == -1
    g.close()


@pytest.mark.parametrize("nx,ny", [(72, 22), (1040, 14), (2048, 10)])
def test_lb_tma_rows_are_bit_identical_to_lb_pull(lb, nx, ny):
    """TMA-staged LB rows (D2Q9 binary32) run the same collision code on the
    same arrived populations as lb_pull: the populations agree bit for bit,
    for a ragged single tile, two full tiles plus a ragged one, and full tiles
    only (halos wrapped periodically at both ends)."""
    p = dict(lattice=9, nx=nx, ny=ny, nz=1, tau=0.8, force=(1e-5, 2e-6, 0.0), precision=1, seed=3)
    a = lb.Lbmpcd(p)
    b = lb.Lbmpcd(p)
    b.set_launch_mode(0, lb_tma=True)
    rng = np.random.default_rng(nx)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f0 = (w[:, None, None] * (1.0 + 0.05 * rng.standard_normal((9, ny, nx)))).ravel()
    a.set("POPS", f0)
    b.set("POPS", f0)
    a.step(70)
    b.step(70)
    np.testing.assert_array_equal(a.get("POPS"), b.get("POPS"))
    np.testing.assert_array_equal(a.get("U"), b.get("U"))
    a.close()
    b.close()


def test_lb_tma_coupled_fp32_matches_oracle(lb):
    """The coupled FP32 step with TMA-staged LB rows against the FP64 oracle
    (1e-5 relative on the populations, 150 steps through two graph chunks)."""
    cfg = inputs.small_2d(precision=1, nx=72)
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    g.set_launch_mode(0, lb_tma=True)
    o = O.OracleSim(dict(cfg["params"], precision=1))
    o.set_region(*cfg["region"])
    g.step(3)
    o.step(3)
    assert rel_err(g.get("POPS"), o.get("POPS")) <= 1e-5
    g.step(147)
    assert np.all(np.isfinite(g.get("POPS")))
    g.close()


def test_barrier_wait_runs_out_and_handle_recovers(lb):
    """A grid-barrier wait that runs out ends the persistent launch with
    ERR_TIMEOUT instead of hanging the GPU: with a poll limit of 1 the first
    block to reach a barrier gives up long before the other (at least one
    per SM) arrive, records the failure, and every other block leaves at its
    next barrier.  With the default limit restored the same handle steps
    again without error, and a fresh handle still matches the oracle."""
    cfg = inputs.small_2d(precision=0, nx=72)
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    g.set_launch_mode(1, 0)
    g.set_wait_limit(1)
    with pytest.raises(lb.LbmpcdError) as ei:
        g.step(4)
    assert ei.value.code == -4   # LBMPCD_ERR_TIMEOUT
    g.set_wait_limit(0)
    g.step(4)
    assert np.all(np.isfinite(g.get("POPS")))
    g.close()
    g = lb.Lbmpcd(cfg["params"])
    o = O.OracleSim(cfg["params"])
    g.set_region(0, *cfg["region"])
    o.set_region(*cfg["region"])
    g.set_launch_mode(1, 0)
    g.step(5)
    o.step(5)
    _check(g, o)
    g.close()
