"""The Chapman-Enskog redraw (redraw = 1) on the GPU: element-wise parity
with the FP64 oracle (the acceptance decisions are taken in binary64 on both
sides), in a sheared channel and from a prescribed non-equilibrium state that
makes most candidates fail; in binary32 the redrawn covariance
(kT/m) I + pi'."""
import math

import numpy as np
import pytest

import oracle as O
from tests import inputs
from tests.test_gpu_parity import FLOOR, lb, pair, rel_err  # noqa: F401
from tests.test_oracle_enskog import _neq_populations

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["2d_shear", "3d_shear", "2d_at", "2d_neq", "3d_neq"])
def test_ce_step_parity_fp64(lb, case):
    over = dict(precision=0, redraw=1)
    if case == "2d_at":
        over["collision"] = 1
    if case.endswith("neq"):
        over.update(kT=1e-3, force=(0, 0, 0))
    cfg = inputs.small_3d(**over) if case.startswith("3d") else inputs.small_2d(**over)
    g, o = pair(lb, cfg)
    p = cfg["params"]
    if case.endswith("neq"):
        Pi0 = np.array([[6e-4, 5e-4, -2e-4], [5e-4, -6e-4, 2.5e-4], [-2e-4, 2.5e-4, 0.0]])
        if case.startswith("2d"):
            Pi0[2] = 0.0
            Pi0[:, 2] = 0.0
        f = _neq_populations(p["lattice"], Pi0, p["nz"], p["ny"], p["nx"]).ravel()
        g.set("POPS", f)
        o.set("POPS", f)
    steps = (1, 1, 3) if case.endswith("neq") else (20, 1, 3)
    for n in steps:
        g.step(n)
        o.step(n)
        assert np.array_equal(g.get("PART_HOME"), o.get("PART_HOME"))
        for fld in ("PART_POS", "PART_VEL", "CELL_VCM", "POPS", "U"):
            e = rel_err(g.get(fld), o.get(fld), FLOOR.get(fld, 0.0))
            assert e <= 1e-12, (fld, e)
    g.close()


def test_ce_redraw_covariance_fp32(lb):
    """Binary32: one step from the prescribed state; peculiar velocities of
    outer-buffer particles away from the walls have covariance
    (kT/m) I + (1 - 1/(2 tau)) Pi0 within 5 standard errors."""
    kT = 1e-3
    cfg = inputs.small_2d(refine=1, ppc=150, kT=kT, alpha=0.0, force=(0, 0, 0), feedback=0, redraw=1, precision=1)
    p = cfg["params"]
    g = lb.Lbmpcd(p)
    g.set_region(0, *cfg["region"])
    Pi0 = np.array([[6e-4, 5e-4, 0], [5e-4, -6e-4, 0], [0, 0, 0]])
    g.set("POPS", _neq_populations(9, Pi0, 1, p["ny"], p["nx"]).ravel())
    home0 = g.get("PART_HOME").reshape(-1, 3)
    g.step(1)
    v = g.get("PART_VEL").reshape(-1, 3)[:, :2]
    x0, x1 = cfg["region"]
    col = x0 + home0[:, 0]
    outer = ((col == x0) | (col == x1 - 1)) & (home0[:, 1] >= 2) & (home0[:, 1] <= p["ny"] - 6)
    C = v[outer]
    want = kT * np.eye(2) + (1 - 1 / (2 * p["tau"])) * Pi0[:2, :2]
    cov = C.T @ C / len(C)
    se = np.sqrt((np.outer(np.diag(want), np.diag(want)) + want ** 2) / len(C))
    print(f"FP32 Chapman-Enskog redraw: covariance {cov.ravel()} want {want.ravel()}")
    assert np.all(np.abs(cov - want) < 5 * se)
    g.close()


def test_ce_restrictions(lb):
    with pytest.raises(lb.LbmpcdError):
        lb.Lbmpcd(inputs.small_2d(redraw=1, precision=2)["params"])
    with pytest.raises(lb.LbmpcdError):
        lb.Lbmpcd(inputs.small_2d(redraw=1, resample_density=1)["params"])
    with pytest.raises(lb.LbmpcdError):
        lb.Lbmpcd(inputs.small_2d(redraw=2)["params"])
    g = lb.Lbmpcd(inputs.small_2d(redraw=1)["params"])
    g.set_region(0, *inputs.small_2d()["region"])
    with pytest.raises(lb.LbmpcdError):
        g.set_launch_mode(1)
    g.close()
