"""Pins of the oracle's coupling: coarse->fine interpolation (Algorithm 2),
LB->MPCD Maxwellian redraw (Sec. 2.3, Algorithm 1), inner-buffer sampling,
the averaging window and the MPCD->LB equilibrium imposition.  Not GPU."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from tests import inputs


def _sim(cfg):
    s = O.OracleSim(cfg["params"])
    s.set_region(*cfg["region"])
    return s


@pytest.mark.parametrize("dim,r", [(2, 1), (2, 2), (2, 4), (3, 2)])
def test_interpolation_reproduces_affine_fields(dim, r):
    """Bilinear/trilinear interpolation is exact on affine fields; with the
    wall ghost u = -u_fluid it is exact on fields vanishing linearly at the
    half-way wall y = 1; at r = 1 it is the identity."""
    cfg = inputs.small_2d(refine=r) if dim == 2 else inputs.small_3d(refine=r)
    p = cfg["params"]
    s = _sim(cfg)
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    x0, x1 = cfg["region"]
    zc, yc, xc = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    A = np.array([[0.3, 0.01, -0.02, 0.005], [-0.1, 0.002, 0.03, -0.004], [0.05, -0.003, 0.001, 0.02]])
    if dim == 2:
        A[:, 3] = 0.0
        A[2] = 0.0
    U = np.stack([a[0] + a[1] * xc + a[2] * yc + a[3] * zc for a in A])
    s.set("U", U)
    Wx, Hy, Wz = (x1 - x0) * r, (ny - 2) * r, (nz * r if dim == 3 else 1)
    for X in range(r, Wx - r):
        for Y in range(r, Hy - r, max(1, Hy // 7)):
            for Z in range(r, max(Wz - r, r + 1), 3) if dim == 3 else [0]:
                px, py = x0 + (X + 0.5) / r, 1 + (Y + 0.5) / r
                pz = (Z + 0.5) / r if dim == 3 else 0.0
                want = A[:, 0] + A[:, 1] * px + A[:, 2] * py + A[:, 3] * pz
                np.testing.assert_allclose(s.u_fine(X, Y, Z), want, atol=1e-13)
    # field (y - 1) * c: exact down to the wall with the ghost rule
    c = np.array([0.02, -0.01, 0.005])
    s.set("U", np.stack([ci * (yc - 1.0) for ci in c]))
    for X in range(r, Wx - r, 2):
        for Y in range(0, Hy // 2):
            np.testing.assert_allclose(s.u_fine(X, Y, r), c * (Y + 0.5) / r, atol=1e-14)
    if r == 1:
        s.set("U", np.random.default_rng(0).normal(size=U.shape))
        U1 = s.get("U").reshape(3, nz, ny, nx)
        for X in range(Wx):
            for Y in range(Hy):
                np.testing.assert_allclose(s.u_fine(X, Y, 0), U1[:, 0, 1 + Y, x0 + X], atol=0)


def test_resample_is_maxwellian_about_lb_velocity():
    """Outer-buffer particles get v = u_LB + sqrt(kT/m) xi, xi ~ N(0, I); the
    rest keep their velocities (alpha = 0 makes the collision the identity)."""
    kT = 4e-4
    cfg = inputs.small_2d(refine=1, ppc=20, kT=kT, alpha=0.0, force=(0, 0, 0), feedback=0)
    s = _sim(cfg)
    zs = []
    for _ in range(4):
        v0 = s.get("PART_VEL").reshape(-1, 3)
        home0 = s.get("PART_HOME").reshape(-1, 3)
        s.step(1)
        v1 = s.get("PART_VEL").reshape(-1, 3)
        x0, x1 = cfg["region"]
        col = x0 + home0[:, 0]
        outer = (col == x0) | (col == x1 - 1)
        # LB at rest (no force, no feedback): u_LB = 0 exactly
        assert np.abs(s.get("U")).max() == 0.0
        zs.append(v1[outer, :2].ravel() / math.sqrt(kT))
        hit = np.any(np.abs(v1[~outer, :2] + v0[~outer, :2]) < 1e-15, axis=1)   # bounce-back flips v
        np.testing.assert_allclose(np.where(hit[:, None], -v1[~outer], v1[~outer]), v0[~outer], atol=1e-15)
    z = np.concatenate(zs)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_sampling_counts_and_momentum():
    """The frame of step 0 holds, per inner-buffer node, exactly the mass of the
    particles whose home cell lies in it, and their mean velocity (pre-collision)."""
    cfg = inputs.small_2d(alpha=0.0, feedback=0, window=1)
    p = cfg["params"]
    s = _sim(cfg)
    s.step(1)
    home = s.get("PART_HOME").reshape(-1, 3)
    v = s.get("PART_VEL").reshape(-1, 3)
    wm = s.get("WINDOW_MEAN").reshape(-1, 4)
    x0, x1 = cfg["region"]
    r, ny = p["refine"], p["ny"]
    col = x0 + home[:, 0] // r
    y = 1 + home[:, 1] // r
    k = 0
    for side, xc in ((0, x0 + 1), (1, x1 - 2)):
        for yy in range(1, ny - 1):
            m = (col == xc) & (y == yy)
            rho_bar = m.sum() * p["mass"] / (p["ppc"] * p["mass"] * r * r)
            assert abs(wm[k, 0] - rho_bar) < 1e-14
            np.testing.assert_allclose(wm[k, 1:3], v[m, :2].mean(0), atol=1e-15)
            k += 1
    assert k == wm.shape[0]


def test_window_is_mean_of_last_W_frames():
    """With window W the imposed moments use the last min(n+1, W) frames:
    mass-weighted velocity, frame-averaged density."""
    base = inputs.small_2d(feedback=0)
    a = _sim(inputs.with_(base, window=1))
    b = _sim(inputs.with_(base, window=3))
    frames = []
    for n in range(6):
        a.step(1)
        b.step(1)
        frames.append(a.get("WINDOW_MEAN").reshape(-1, 4))
        last = frames[-3:]
        rho = np.mean([f[:, 0] for f in last], axis=0)
        mom = np.sum([f[:, 0:1] * f[:, 1:] for f in last], axis=0)
        want_u = mom / np.sum([f[:, 0:1] for f in last], axis=0)
        wb = b.get("WINDOW_MEAN").reshape(-1, 4)
        np.testing.assert_allclose(wb[:, 0], rho, rtol=1e-13)
        np.testing.assert_allclose(wb[:, 1:], want_u, rtol=1e-11, atol=1e-16)


def test_imposition_writes_equilibrium_of_window_mean():
    """The window mean a8 records at step n is imposed by the LB update of
    step n + 1: the inner-buffer populations after that update are f_eq
    (Eq. 2) at the node's LB density of step n + 1 and the window-mean MPCD
    velocity of step n, so their zeroth and first moments are rho_LB and
    rho_LB u_bar.  Nothing is imposed from the window of step 0, so the first
    imposed populations are those after step 2."""
    cfg = inputs.small_2d(feedback=1, window=3)
    p = cfg["params"]
    s = _sim(cfg)
    x0, x1 = cfg["region"]
    ny, nx = p["ny"], p["nx"]
    c, _ = O.lattice(9)
    wm_prev = None
    for n in range(4):
        s.step(1)
        f = s.get("POPS").reshape(9, ny, nx)
        rho = s.get("RHO").reshape(ny, nx)
        k = 0
        for xc in (x0 + 1, x1 - 2):
            for yy in range(1, ny - 1):
                if n >= 2:
                    want = O.feq(9, rho[yy, xc], wm_prev[k, 1:3])
                    assert abs(f[:, yy, xc].sum() - rho[yy, xc]) < 1e-14
                    np.testing.assert_allclose(f[:, yy, xc] @ c[:, :2], rho[yy, xc] * wm_prev[k, 1:3], atol=1e-16)
                    np.testing.assert_allclose(f[:, yy, xc], want, rtol=0, atol=1e-15)
                elif n == 1:
                    want = O.feq(9, rho[yy, xc], wm_prev[k, 1:3])
                    assert np.max(np.abs(f[:, yy, xc] - want)) > 1e-6
                k += 1
        wm_prev = s.get("WINDOW_MEAN").reshape(-1, 4)


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_one_way_coupling_leaves_lb_untouched(case):
    """feedback = 0 is the paper's one-way coupling: the LB populations are
    bit-identical to an LB-only run."""
    cfg = inputs.small_2d(feedback=0) if case == "2d" else inputs.small_3d(feedback=0)
    a = _sim(cfg)
    b = O.OracleSim(cfg["params"])
    a.step(4)
    b.step(4)
    assert np.array_equal(a.get("POPS"), b.get("POPS"))


def test_particle_count_and_bounds_conserved():
    """Periodic wrap in the region keeps the particle number fixed (NVT, Sec. 2.3)
    and every particle inside the region."""
    cfg = inputs.small_3d()
    s = _sim(cfg)
    n0 = s.num_particles
    s.step(5)
    home = s.get("PART_HOME").reshape(-1, 3)
    off = s.get("PART_POS").reshape(-1, 3)
    p = cfg["params"]
    r = p["refine"]
    assert s.get("DIAG")[4] == n0
    assert home[:, 0].min() >= 0 and home[:, 0].max() < (cfg["region"][1] - cfg["region"][0]) * r
    assert home[:, 1].min() >= 0 and home[:, 1].max() < (p["ny"] - 2) * r
    assert home[:, 2].min() >= 0 and home[:, 2].max() < p["nz"] * r
    assert off.min() >= 0 and off.max() < 1


@pytest.mark.slow
def test_two_way_coupling_stays_bounded():
    """With the windowed feedback the coupled channel stays at the noise level:
    over 1500 steps the LB speed stays below 1e-2 and rho within 1 %."""
    cfg = inputs.small_2d(refine=2, ppc=10, tau=0.8, force=(1e-7, 0, 0), kT=1e-4, window=100,
                          nx=128, ny=34)
    cfg["region"] = (48, 80)
    s = _sim(cfg)
    for _ in range(3):
        s.step(500)
        u = s.get("U")
        rho = s.get("RHO").reshape(34, 128)[1:-1]
        assert np.all(np.isfinite(u)) and np.abs(u).max() < 1e-2
        assert np.abs(rho - 1).max() < 1e-2
