"""Pins of the oracle's lattice Boltzmann step (Eq. 1-2, Sec. 2.1, Sec. 3)."""
import numpy as np
import pytest

import oracle as O
from tests import inputs


@pytest.mark.parametrize("lat,dim", [(9, 2), (19, 3)])
def test_lattice_isotropy(lat, dim):
    """sum w = 1, sum w c c = cs^2 I, sum w c^4 = cs^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)."""
    c, w = O.lattice(lat)
    c = c[:, :dim].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(dim) / 3.0, atol=1e-15)
    d = np.eye(dim)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-15)
    # every velocity has its opposite
    for ci in c:
        assert any(np.array_equal(-ci, cj) for cj in c)


@pytest.mark.parametrize("lat,dim", [(9, 2), (19, 3)])
def test_feq_moments(lat, dim):
    """Eq. 2 has moments rho, rho u and rho (cs^2 I + u u) (Sec. 2.1)."""
    c, _ = O.lattice(lat)
    c = c[:, :dim].astype(float)
    rng = np.random.default_rng(5)
    for _ in range(20):
        rho = rng.uniform(0.5, 1.5)
        u = rng.uniform(-0.1, 0.1, size=dim)
        f = O.feq(lat, rho, u)
        assert abs(f.sum() - rho) < 1e-14
        np.testing.assert_allclose(f @ c, rho * u, atol=1e-15)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f, c, c),
                                   rho * (np.eye(dim) / 3.0 + np.outer(u, u)), atol=1e-14)


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_lb_mass_conserved(case):
    """Bounce-back walls, periodic x/z and the Guo force conserve LB mass exactly."""
    cfg = inputs.small_2d() if case == "2d" else inputs.small_3d()
    p = dict(cfg["params"])
    s = O.OracleSim(p)
    c, w = O.lattice(p["lattice"])
    f0 = inputs.perturbed_populations(len(w), (p["nz"], p["ny"], p["nx"]), w, seed=3, amp=0.05)
    s.set("POPS", f0)
    m0 = s.get("DIAG")[0]
    s.step(40)
    m1 = s.get("DIAG")[0]
    assert abs(m1 - m0) <= 1e-13 * m0


def _poiseuille(lat, tau, H, g, axis=0, nz=1, steps=3000):
    ny = H + 2
    force = [0.0, 0.0, 0.0]
    force[axis] = g
    s = O.OracleSim(dict(lattice=lat, nx=3, ny=ny, nz=nz, tau=tau, force=force))
    s.step(steps)
    u = s.get("U").reshape(3, nz, ny, 3)[axis, 0, 1:-1, 1]
    y = np.arange(1, ny - 1) + 0.5 - 1.0          # distance from the half-way wall
    return y, u


@pytest.mark.parametrize("lat,nz,axis", [(9, 1, 0), (19, 2, 0), (19, 2, 2)])
def test_poiseuille_exact_at_magic_tau(lat, nz, axis):
    """At (tau-1/2)^2 = 3/16 BGK with half-way bounce-back reproduces the
    parabola u = g y (H - y) / (2 nu), nu = cs^2 (tau - 1/2) (Sec. 2.1), exactly."""
    tau = 0.5 + np.sqrt(3.0) / 4.0
    H, g = 8, 1e-5
    y, u = _poiseuille(lat, tau, H, g, axis=axis, nz=nz, steps=2500)
    nu = (tau - 0.5) / 3.0
    ua = g * y * (H - y) / (2 * nu)
    assert np.max(np.abs(u - ua)) < 1e-9 * ua.max()


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.5])
def test_poiseuille_curvature_and_slip(tau):
    """Steady BGK Poiseuille: curvature -g/nu exactly, and the known half-way
    bounce-back slip u_s = g (16 L - 3) / (24 nu), L = (tau - 1/2)^2
    (He, Zou, Luo, Dembo 1997; Ginzburg & d'Humieres 2003)."""
    H, g = 8, 1e-5
    nu = (tau - 0.5) / 3.0
    steps = int(40 * H * H / (np.pi ** 2 * nu)) + 200
    y, u = _poiseuille(9, tau, H, g, steps=steps)
    coef = np.polyfit(y, u, 2)
    assert abs(2 * coef[0] + g / nu) < 1e-8 * g / nu
    lam = (tau - 0.5) ** 2
    slip = g * (16 * lam - 3) / (24 * nu)
    np.testing.assert_allclose(u, g * y * (H - y) / (2 * nu) + slip, rtol=0, atol=1e-9 * u.max())


def _startup_series(y, t, H, g, nu, terms=400):
    """Plane Poiseuille flow started from rest: the steady parabola minus the
    decaying odd sine modes, y from the wall."""
    u = g * y * (H - y) / (2 * nu)
    for n in range(1, 2 * terms, 2):
        u -= 4 * g * H * H / (nu * np.pi ** 3 * n ** 3) * np.sin(n * np.pi * y / H) * np.exp(-(n * np.pi / H) ** 2 * nu * t)
    return u


@pytest.mark.parametrize("lat,nz", [(9, 1), (19, 2)])
def test_poiseuille_startup_follows_the_series_solution(lat, nz):
    """From rest under a constant force the LB profile follows the transient
    series solution (Sec. 3's Poiseuille benchmark before it is steady):
    after n steps, n = 100 .. 800 with H^2 / nu = 2770, within 0.1% of the
    centreline value, the velocity with the half-force shift being that of
    time n - 1/2 (at (tau - 1/2)^2 = 3/16, where the walls sit exactly half
    way).  A viscosity 5% off misses by 0.8% or more."""
    tau = 0.5 + np.sqrt(3.0) / 4.0
    nu = (tau - 0.5) / 3.0
    H, g = 20, 1e-6
    ny = H + 2
    s = O.OracleSim(dict(lattice=lat, nx=3, ny=ny, nz=nz, tau=tau, force=(g, 0.0, 0.0)))
    y = np.arange(1, ny - 1) + 0.5 - 1.0
    done = 0
    for t in (100, 200, 400, 800):
        s.step(t - done)
        done = t
        u = s.get("U").reshape(3, nz, ny, 3)[0, 0, 1:-1, 1]
        ua = _startup_series(y, t - 0.5, H, g, nu)
        assert np.max(np.abs(u - ua)) < 1e-3 * ua.max(), (t, np.max(np.abs(u - ua)) / ua.max())
