"""MPCD-AT collisions (Eq. 6, collision = 1) on the GPU against the FP64
oracle: single steps element by element (1e-12 in FP64, 1e-5 in FP32 away
from cell edges), through graph chunks with their particle sort, and the
argument checks of the mode."""
import numpy as np
import pytest

from tests import inputs
from tests.test_gpu_parity import FLOOR, ambiguous_particles, lb, pair, rel_err  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["2d", "3d", "2d_r1", "2d_oneway", "2d_hot"])
def test_at_step_parity_fp64(lb, case):
    over = dict(precision=0, collision=1)
    if case == "2d_r1":
        over["refine"] = 1
    if case == "2d_oneway":
        over["feedback"] = 0
    if case == "2d_hot":
        over.update(kT=0.01, mass=2.0)
    cfg = inputs.small_3d(**over) if case == "3d" else inputs.small_2d(**over)
    g, o = pair(lb, cfg)
    for n in (1, 1, 3):
        g.step(n)
        o.step(n)
        assert np.array_equal(g.get("SHIFT"), o.get("SHIFT"))
        assert np.array_equal(g.get("PART_HOME"), o.get("PART_HOME"))
        assert np.array_equal(g.get("PART_CELL"), o.get("PART_CELL"))
        assert np.array_equal(g.get("CELL_COUNT"), o.get("CELL_COUNT"))
        for f in ("PART_POS", "PART_VEL", "CELL_VCM", "WINDOW_MEAN", "POPS", "RHO", "U"):
            e = rel_err(g.get(f), o.get(f), FLOOR.get(f, 0.0))
            assert e <= 1e-12, (f, e)
        np.testing.assert_allclose(g.get("DIAG"), o.get("DIAG"), rtol=1e-12, atol=1e-13)
    g.close()


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_at_run_with_sorting_fp64(lb, case):
    """150 steps: two 64-step graph chunks with the sort (the stored random
    velocities move with their particles) and a remainder."""
    over = dict(precision=0, collision=1)
    cfg = inputs.small_2d(nx=72, **over) if case == "2d" else inputs.small_3d(nx=24, **over)
    g, o = pair(lb, cfg)
    g.step(150)
    o.step(150)
    assert np.array_equal(g.get("PART_HOME"), o.get("PART_HOME"))
    assert np.array_equal(g.get("PART_CELL"), o.get("PART_CELL"))
    for f in ("PART_POS", "PART_VEL", "CELL_VCM", "WINDOW_MEAN", "POPS", "U"):
        e = rel_err(g.get(f), o.get(f), FLOOR.get(f, 0.0))
        assert e <= 1e-12, (f, e)
    g.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_at_step_parity_fp32(lb, dim):
    """Binary32 storage and arithmetic (binary32 Box-Muller) against the FP64
    oracle: 1e-5 relative away from cell edges."""
    cfg = inputs.small_2d(precision=1, collision=1) if dim == 2 else inputs.small_3d(precision=1, collision=1)
    g, o = pair(lb, cfg)
    for n in (1, 2):
        g.step(n)
        o.step(n)
        amb = ambiguous_particles(o, dim, 1e-5)
        cells_o, cells_g = o.get("PART_CELL"), g.get("PART_CELL")
        bad = set(cells_o[amb]) | set(cells_g[amb])
        ok = ~np.isin(cells_o, list(bad)) & ~amb
        assert ok.mean() > 0.9
        assert np.array_equal(cells_g[ok], cells_o[ok])
        vg = g.get("PART_VEL").reshape(-1, 3)[ok]
        vo = o.get("PART_VEL").reshape(-1, 3)[ok]
        assert rel_err(vg, vo) <= 1e-5
        for f in ("POPS", "RHO", "U"):
            assert rel_err(g.get(f), o.get(f), FLOOR.get(f, 0.0)) <= 1e-5, f
    g.close()


def test_at_fp16_storage_runs(lb):
    """MPCD-AT with binary16 LB storage (particles in binary32): a sorted chunk
    plus a remainder stays finite and keeps every particle and the cell sums."""
    cfg = inputs.small_2d(precision=2, collision=1, nx=72)
    g = lb.Lbmpcd(cfg["params"])
    g.set_region(0, *cfg["region"])
    n0 = g.get("PART_ID").size
    g.step(70)
    v = g.get("PART_VEL")
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(g.get("POPS")))
    cells, cnt = g.get("PART_CELL"), g.get("CELL_COUNT")
    assert cells.size == n0 and np.array_equal(np.bincount(cells, minlength=cnt.size), cnt)
    g.close()


def test_at_mode_restrictions(lb):
    with pytest.raises(lb.LbmpcdError) as ei:
        lb.Lbmpcd(inputs.small_2d(collision=1, resample_density=1)["params"])
    assert ei.value.code == -1
    with pytest.raises(lb.LbmpcdError):
        lb.Lbmpcd(inputs.small_2d(collision=2)["params"])
    mixed = [inputs.small_2d()["params"], inputs.small_2d(collision=1)["params"]]
    with pytest.raises(lb.LbmpcdError):
        lb.Lbmpcd(mixed)
    g = lb.Lbmpcd(inputs.small_2d(collision=1)["params"])
    g.set_region(0, *inputs.small_2d()["region"])
    with pytest.raises(lb.LbmpcdError):
        g.set_launch_mode(1)                       # no persistent form for MPCD-AT
    choice = g.autotune(steps=8)
    assert choice["mode"] == 0
    g.step(3)
    assert np.all(np.isfinite(g.get("PART_VEL")))
    g.close()
