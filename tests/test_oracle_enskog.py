"""Pins of the oracle's Chapman-Enskog redraw (redraw = 1; the Enskog sampling
Sec. 2.3 names for strong gradients): the LB's non-equilibrium momentum flux
against the momentum balance of a Poiseuille flow, and the redrawn peculiar
velocities' covariance (kT/m) I + pi' against a prescribed non-equilibrium
state.  Not GPU."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from tests import inputs

CS2 = 1.0 / 3.0


def _neq_populations(lat, Pi0, nz, ny, nx):
    """Uniform f = f_eq(1, 0) + w_i Q_i : Pi0 / (2 cs^4), Q_i = c_i c_i - cs^2 I:
    zero mass and momentum, second moment Pi0 (lattice isotropy)."""
    c, w = O.lattice(lat)
    f = O.feq(lat, 1.0, [0.0, 0.0, 0.0])
    Q = np.einsum("ia,ib->iab", c, c) - CS2 * np.eye(3)[None]
    fneq = w * np.einsum("iab,ab->i", Q, Pi0) / (2 * CS2 * CS2)
    assert abs(fneq.sum()) < 1e-15 and np.abs(fneq @ c).max() < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", fneq, c, c), Pi0, atol=1e-15)
    return np.broadcast_to((f + fneq)[:, None, None, None], (len(f), nz, ny, nx)).copy()


def test_pi_of_poiseuille_balances_the_body_force():
    """Steady Poiseuille: the shear component of the kinematic momentum flux
    carries the force, pi_xy(y) = -g (ny/2 - y) (y at node centres, walls
    half-way), whatever nu; the normal components vanish."""
    g, ny, nx, tau = 1e-5, 22, 4, 0.5 + math.sqrt(3.0) / 4.0
    p = dict(lattice=9, nx=nx, ny=ny, nz=1, tau=tau, force=(g, 0, 0), redraw=1)
    s = O.OracleSim(p)
    nu = (tau - 0.5) / 3.0
    yc = np.arange(ny) + 0.5
    u = np.where((yc > 1) & (yc < ny - 1), g * (yc - 1) * (ny - 1 - yc) / (2 * nu), 0.0)
    f = np.stack([O.feq(9, 1.0, [ui, 0.0, 0.0]) for ui in u])
    s.set("POPS", np.repeat(f.T[:, :, None], nx, axis=2).ravel())
    s.step(3000)
    pi = s.get("PI").reshape(6, ny, nx)[:, 1:-1, 0]
    want = -g * (ny / 2.0 - yc[1:-1])
    np.testing.assert_allclose(pi[3], want, rtol=0, atol=2e-3 * g * ny / 2)
    assert np.abs(pi[0]).max() < 1e-3 * g * ny / 2 and np.abs(pi[0] + pi[1]).max() < 1e-18


@pytest.mark.parametrize("dim", [2, 3])
def test_ce_redraw_covariance(dim):
    """One step from a uniform non-equilibrium state with second moment Pi0:
    the redrawn peculiar velocities of outer-buffer particles away from the
    walls have covariance (kT/m) I + (1 - 1/(2 tau)) Pi0' (alpha = 0 keeps them
    through the collision, no force, u_LB = 0)."""
    kT = 1e-3
    if dim == 2:
        cfg = inputs.small_2d(refine=1, ppc=150, kT=kT, alpha=0.0, force=(0, 0, 0), feedback=0, redraw=1)
        Pi0 = np.array([[6e-4, 5e-4, 0], [5e-4, -6e-4, 0], [0, 0, 0]])
    else:
        cfg = inputs.small_3d(refine=1, ppc=60, kT=kT, alpha=0.0, force=(0, 0, 0), feedback=0, redraw=1)
        Pi0 = np.array([[4e-4, 3e-4, -2e-4], [3e-4, -1e-4, 2.5e-4], [-2e-4, 2.5e-4, -3e-4]])
    p = cfg["params"]
    s = O.OracleSim(p)
    s.set_region(*cfg["region"])
    lat, nz, ny, nx = p["lattice"], p["nz"], p["ny"], p["nx"]
    s.set("POPS", _neq_populations(lat, Pi0, nz, ny, nx).ravel())
    home0 = s.get("PART_HOME").reshape(-1, 3)
    s.step(1)
    v = s.get("PART_VEL").reshape(-1, 3)[:, :dim]
    x0, x1 = cfg["region"]
    col = x0 + home0[:, 0]
    outer = ((col == x0) | (col == x1 - 1)) & (home0[:, 1] >= 2) & (home0[:, 1] <= ny - 6)
    C = v[outer]
    assert np.abs(s.get("U")).max() < 1e-15
    want = kT * np.eye(dim) + (1 - 1 / (2 * p["tau"])) * Pi0[:dim, :dim]
    cov = C.T @ C / len(C)
    # standard error of a sample second moment: sqrt((<x^2><y^2> + <xy>^2) / N)
    se = np.sqrt((np.outer(np.diag(want), np.diag(want)) + want ** 2) / len(C))
    assert len(C) > 4000
    assert np.all(np.abs(cov - want) < 5 * se), (cov, want)
    assert np.abs(C.mean(0)).max() < 5 * math.sqrt(kT / len(C))


def test_ce_redraw_without_stress_is_maxwellian():
    """LB at rest: b = 0, every first candidate is accepted and the peculiar
    velocities are N(0, kT/m)."""
    kT = 4e-4
    cfg = inputs.small_2d(refine=1, ppc=20, kT=kT, alpha=0.0, force=(0, 0, 0), feedback=0, redraw=1)
    s = O.OracleSim(cfg["params"])
    s.set_region(*cfg["region"])
    home0 = s.get("PART_HOME").reshape(-1, 3)
    s.step(1)
    v = s.get("PART_VEL").reshape(-1, 3)
    x0, x1 = cfg["region"]
    col = x0 + home0[:, 0]
    outer = (col == x0) | (col == x1 - 1)
    assert np.abs(s.get("PI")).max() == 0.0
    z = v[outer, :2].ravel() / math.sqrt(kT)     # a wall bounce flips the sign: still N(0, 1)
    assert stats.kstest(z, "norm").pvalue > 1e-4


@pytest.mark.parametrize("over", [dict(redraw=2), dict(redraw=-1), dict(redraw=1, resample_density=1)])
def test_redraw_mode_is_validated(over):
    with pytest.raises(ValueError):
        O.OracleSim(inputs.small_2d(**over)["params"])
