"""Pins of the oracle's near-wall strip (the two-level geometry of Sec. 3.3):
the MPCD region spans all columns and the LB rows [1, y1) next to the bottom
wall, with the coupling buffer along its top edge (outer rows redrawn from the
LB, inner rows sampled and imposed), a specular top edge and no virtual
particles there.  Not GPU."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle as O
from oracle import transport as T
from tests import inputs

DEG = math.pi / 180.0


def _strip(cfg, y1):
    s = O.OracleSim(cfg["params"])
    s.set_strip(y1)
    return s


def _flight(home, off, vel):
    """One particle among resting ones in a 4-column strip of Hs = 4 rows
    (ny = 8, y1 = 5, no buffer, kT = 0, alpha = 0)."""
    p = dict(lattice=9, nx=4, ny=8, nz=1, tau=1.0, force=(0, 0, 0), refine=1, ppc=3, alpha=0.0, kT=0.0,
             coupling_width=0, feedback=0, seed=5)
    s = O.OracleSim(p)
    s.set_strip(5)
    H = s.get("PART_HOME").reshape(-1, 3)
    X = s.get("PART_POS").reshape(-1, 3)
    V = np.zeros((s.num_particles, 3))
    H[0, :2], X[0, :2], V[0, :2] = home, off, vel
    s.set("PART_HOME", H.ravel())
    s.set("PART_POS", X.ravel())
    s.set("PART_VEL", V.ravel())
    s.step(1)
    return s.get("PART_HOME").reshape(-1, 3)[0], s.get("PART_POS").reshape(-1, 3)[0], s.get("PART_VEL").reshape(-1, 3)[0]


def _exact(X0, Y0, vx, vy, Hs, W):
    """Straight flight; at y = 0 (wall) the velocity reverses (bounce-back), at
    y = Hs (the strip's top edge) only v_y does (specular)."""
    X0, Y0, vx, vy = map(Fraction, (X0, Y0, vx, vy))
    Y1 = Y0 + vy
    if 0 <= Y1 < Hs:
        return (X0 + vx) % W, Y1, vx, vy
    if Y1 >= Hs:
        return (X0 + vx) % W, Hs - (Y1 - Hs), vx, -vy
    ts = -Y0 / vy
    Xh = X0 + vx * ts
    return (Xh - vx * (1 - ts)) % W, -vy * (1 - ts), -vx, -vy


@pytest.mark.parametrize("home,off,vel", [
    ((1, 3), (0.5, 0.75), (0.2, 0.5)),      # crosses the top edge: specular
    ((2, 3), (0.25, 0.875), (-0.375, 0.25)),  # top edge, moving left, wraps nothing
    ((3, 0), (0.9, 0.25), (0.3, -0.5)),      # bottom wall: bounce-back, x wrap
    ((0, 2), (0.05, 0.5), (-0.2, 0.25)),     # interior, wraps in x
])
def test_strip_streaming_matches_exact_flight(home, off, vel):
    h, o, v = _flight(home, off, vel)
    Xe, Ye, vxe, vye = _exact(home[0] + off[0], home[1] + off[1], vel[0], vel[1], 4, 4)
    assert abs((h[0] + o[0]) - float(Xe)) < 1e-14 and abs((h[1] + o[1]) - float(Ye)) < 1e-14
    assert 0 <= h[1] < 4 and 0 <= o[0] < 1 and 0 <= o[1] < 1
    np.testing.assert_allclose(v[:2], [float(vxe), float(vye)], atol=1e-15)


def test_strip_outer_rows_are_redrawn():
    """Particles in the top LB row of the strip get u_LB + sqrt(kT/m) xi; the
    others keep their velocities (alpha = 0; bounce-back at the bottom wall
    flips them)."""
    kT = 4e-4
    cfg = inputs.small_2d(refine=1, ppc=20, kT=kT, alpha=0.0, force=(0, 0, 0), feedback=0)
    y1 = 8
    s = _strip(cfg, y1)
    zs = []
    for _ in range(4):
        v0 = s.get("PART_VEL").reshape(-1, 3)
        home0 = s.get("PART_HOME").reshape(-1, 3)
        s.step(1)
        v1 = s.get("PART_VEL").reshape(-1, 3)
        outer = 1 + home0[:, 1] == y1 - 1
        assert np.abs(s.get("U")).max() == 0.0
        zs.append(v1[outer, :2].ravel() / math.sqrt(kT))
        hit = np.any(np.abs(v1[~outer, :2] + v0[~outer, :2]) < 1e-15, axis=1)
        np.testing.assert_allclose(np.where(hit[:, None], -v1[~outer], v1[~outer]), v0[~outer], atol=1e-15)
    assert stats.kstest(np.concatenate(zs), "norm").pvalue > 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_strip_sampling_counts_and_momentum(dim):
    """Frame of step 0, W = 1: per node of the inner row (y1 - 2 for a 2-row
    buffer), the mass and mean velocity of the particles whose home cell lies
    in it; entries ordered (row, z, x)."""
    cfg = (inputs.small_2d if dim == 2 else inputs.small_3d)(alpha=0.0, feedback=0, window=1)
    p = cfg["params"]
    y1 = 6
    s = _strip(cfg, y1)
    s.step(1)
    home = s.get("PART_HOME").reshape(-1, 3)
    v = s.get("PART_VEL").reshape(-1, 3)
    wm = s.get("WINDOW_MEAN").reshape(-1, 4)
    r, nx, nz = p["refine"], p["nx"], p["nz"]
    assert wm.shape[0] == nx * nz
    x, y, z = home[:, 0] // r, 1 + home[:, 1] // r, home[:, 2] // r
    rd = r ** dim
    for zz in range(nz):
        for xx in range(nx):
            m = (x == xx) & (y == y1 - 2) & (z == zz)
            k = zz * nx + xx
            assert abs(wm[k, 0] - m.sum() / (p["ppc"] * rd)) < 1e-14
            np.testing.assert_allclose(wm[k, 1:1 + dim], v[m, :dim].mean(0), atol=1e-15)


def test_strip_imposition_on_the_inner_row():
    """feedback = 1: the window mean of step n is imposed on the inner row by
    the LB update of step n + 1 (from the window of step 1 on): f_eq(rho_LB,
    u_bar); no other row is touched by it."""
    cfg = inputs.small_2d(feedback=1, window=3)
    p = cfg["params"]
    ny, nx = p["ny"], p["nx"]
    y1 = 7
    s = _strip(cfg, y1)
    c, _ = O.lattice(9)
    wm_prev = None
    for n in range(4):
        s.step(1)
        f = s.get("POPS").reshape(9, ny, nx)
        rho = s.get("RHO").reshape(ny, nx)
        for xx in range(0, nx, 5):
            if n >= 2:
                want = O.feq(9, rho[y1 - 2, xx], wm_prev[xx, 1:3])
                np.testing.assert_allclose(f[:, y1 - 2, xx], want, rtol=0, atol=1e-15)
                np.testing.assert_allclose(f[:, y1 - 2, xx] @ c[:, :2], rho[y1 - 2, xx] * wm_prev[xx, 1:3],
                                           atol=1e-16)
            elif n == 1:
                want = O.feq(9, rho[y1 - 2, xx], wm_prev[xx, 1:3])
                assert np.max(np.abs(f[:, y1 - 2, xx] - want)) > 1e-6
        wm_prev = s.get("WINDOW_MEAN").reshape(-1, 4)


@pytest.mark.parametrize("dim", [2, 3])
def test_strip_one_way_leaves_lb_untouched_and_keeps_particles(dim):
    cfg = (inputs.small_2d if dim == 2 else inputs.small_3d)(feedback=0)
    p = cfg["params"]
    y1 = 6
    a = _strip(cfg, y1)
    b = O.OracleSim(p)
    n0 = a.num_particles
    a.step(5)
    b.step(5)
    assert np.array_equal(a.get("POPS"), b.get("POPS"))
    home = a.get("PART_HOME").reshape(-1, 3)
    r = p["refine"]
    assert a.get("DIAG")[4] == n0 == p["nx"] * r * (y1 - 1) * r * (p["nz"] * r if dim == 3 else 1) * p["ppc"]
    assert home[:, 1].min() >= 0 and home[:, 1].max() < (y1 - 1) * r
    assert home[:, 0].max() < p["nx"] * r


def test_strip_top_cells_get_no_virtual_particles():
    """SRD conserves the momentum of every cell but the bottom wall's cut cells:
    the cells cut by the strip's top edge take no virtual particles."""
    base = dict(lattice=9, nx=16, ny=12, nz=1, tau=1.0, force=(0, 0, 0), refine=1, ppc=6, kT=1e-3,
                coupling_width=0, feedback=0, seed=9)
    a = O.OracleSim(dict(base, alpha=130 * DEG))
    b = O.OracleSim(dict(base, alpha=0.0))
    a.set_strip(8)
    b.set_strip(8)
    Hs = 7
    top_checked = 0
    for _ in range(4):
        a.step(1)
        b.step(1)
        cells = a.get("PART_CELL")
        va, vb = a.get("PART_VEL").reshape(-1, 3), b.get("PART_VEL").reshape(-1, 3)
        cy = cells // 16
        for c in np.unique(cells[cy > 0]):
            m = cells == c
            np.testing.assert_allclose(va[m].sum(0), vb[m].sum(0), rtol=0, atol=1e-15)
            top_checked += (c // 16 == Hs) and m.sum() < 6
        b.set("PART_VEL", va.ravel())
    assert top_checked > 0


def test_near_wall_poiseuille_sec33():
    """Sec. 3.3: an MPCD-AT strip of 8 rows at the bottom wall of a 20-node
    Poiseuille channel, one-way coupled (feedback 0), viscosity matched by
    Eq. 7 (nu = 1/6, tau = 1); LB started on the steady profile.  The strip's
    time-averaged profile (4000 steps after 1000) follows the analytic
    u = g (y - 1)(ny - 1 - y) / (2 nu) within 6% L2 (measured 3.1%)."""
    nx, ny, y1, ppc, g, nu = 20, 22, 9, 10, 3e-4, 1.0 / 6.0
    kT = T.at_kT_for_viscosity(nu, ppc, 1.0)
    p = dict(lattice=9, nx=nx, ny=ny, nz=1, tau=1.0, force=(g, 0, 0), refine=1, ppc=ppc, alpha=0.0, kT=kT,
             mass=1.0, coupling_width=2, precision=0, feedback=0, window=1, seed=3, collision=1)
    s = O.OracleSim(p)
    s.set_strip(y1)
    yc = np.arange(ny) + 0.5
    u = np.where((yc > 1) & (yc < ny - 1), g * (yc - 1) * (ny - 1 - yc) / (2 * nu), 0.0)
    f = np.stack([O.feq(9, 1.0, [ui, 0.0, 0.0]) for ui in u])
    s.set("POPS", np.repeat(f.T[:, :, None], nx, axis=2).ravel())
    s.step(1000)
    Hs = y1 - 1
    mom, cnt = np.zeros(Hs), np.zeros(Hs)
    for _ in range(4000):
        s.step(1)
        h = s.get("PART_HOME").reshape(-1, 3)
        v = s.get("PART_VEL").reshape(-1, 3)
        mom += np.bincount(h[:, 1], weights=v[:, 0], minlength=Hs)
        cnt += np.bincount(h[:, 1], minlength=Hs)
    y = 1.0 + np.arange(Hs) + 0.5
    ua = g * (y - 1) * (ny - 1 - y) / (2 * nu)
    err = np.linalg.norm(mom / cnt - ua) / np.linalg.norm(ua)
    print(f"near-wall strip: rel. L2 against the analytic profile {err:.4f}")
    assert err < 0.06


@pytest.mark.parametrize("y1,over", [(3, {}), (21, {}), (8, dict(feedback=2)), (8, dict(resample_density=1))])
def test_strip_is_validated(y1, over):
    cfg = inputs.small_2d(**over)
    s = O.OracleSim(cfg["params"])
    with pytest.raises(ValueError):
        s.set_strip(y1)
