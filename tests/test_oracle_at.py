"""Pins of the oracle's MPCD-AT collision (Eq. 6, collision = 1): the cell
momentum is kept, the relative velocities are replaced by thermal ones of
variance kT/m (whatever they were), virtual wall particles take part with the
right weight, and Eq. 7 solved for kT gives the thermal energies Table 1
prints.  The viscosity itself is pinned in test_oracle_viscosity.py.  Not GPU."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O
from oracle import transport as T

DEG = math.pi / 180.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_mpcd_at.txt")


def toy(dim=2, **over):
    """A small box with walls in y, no LB force, no coupling buffer."""
    if dim == 2:
        p = dict(lattice=9, nx=16, ny=10, nz=1, tau=1.0, force=(0, 0, 0), refine=1, ppc=6,
                 alpha=130 * DEG, kT=1e-3, coupling_width=0, feedback=0, seed=17, collision=1)
    else:
        p = dict(lattice=19, nx=8, ny=8, nz=6, tau=1.0, force=(0, 0, 0), refine=1, ppc=5,
                 alpha=120 * DEG, kT=1e-3, coupling_width=0, feedback=0, seed=17, collision=1)
    p.update(over)
    s = O.OracleSim(p)
    s.set_region(0, p["nx"])
    return s, p


def _pair(dim, **over):
    """An MPCD-AT system and the same system under SRD with alpha = 0, whose
    post-collision velocities are the pre-collision ones."""
    a, p = toy(dim, **over)
    b, _ = toy(dim, collision=0, alpha=0.0, **over)
    return a, b, p


def _cut_mask(cells, p, shift_y):
    ncx, ncy = p["nx"] * p["refine"], (p["ny"] - 2) * p["refine"] + 1
    cy = (cells // ncx) % ncy
    return ((cy == 0) | (cy == ncy - 1)) & (shift_y > 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_at_keeps_cell_momentum_not_energy(dim):
    """Eq. 6 adds v_ran - <v_ran> to v_cm: the cell momentum is unchanged in
    every cell without virtual particles, the kinetic energy is not (the
    collision is a thermostat)."""
    a, b, p = _pair(dim)
    changed = 0
    for _ in range(3):
        a.step(1)
        b.step(1)
        cells = a.get("PART_CELL")
        assert np.array_equal(cells, b.get("PART_CELL"))
        va = a.get("PART_VEL").reshape(-1, 3)
        vb = b.get("PART_VEL").reshape(-1, 3)
        cut = _cut_mask(cells, p, a.get("SHIFT")[1])
        for c in np.unique(cells[~cut]):
            m = cells == c
            np.testing.assert_allclose(va[m].sum(0), vb[m].sum(0), rtol=0, atol=1e-15)
            if m.sum() > 1:
                changed += abs((va[m] ** 2).sum() - (vb[m] ** 2).sum()) > 1e-3 * (vb[m] ** 2).sum()
        b.set("PART_VEL", va.ravel())          # keep the two runs in step
    assert changed > 10


@pytest.mark.parametrize("dim", [2, 3])
def test_at_replaces_relative_velocities_by_thermal_ones(dim):
    """Pre-collision velocities 10x hotter than kT: after one collision the
    relative velocities in a cell of n particles carry (kT/m) chi^2 with
    d (n - 1) degrees of freedom in total (Eq. 6 with variance kT/m per
    component, Algorithm 1), whatever they were before; m = 2 so that kT and
    kT/m differ."""
    kT, m = 0.01, 2.0
    big = {2: dict(nx=24, ny=26, ppc=8), 3: dict(nx=12, ny=14, nz=12, ppc=6)}[dim]
    s, p = toy(dim, kT=kT, mass=m, **big)
    rng = np.random.default_rng(3)
    v = rng.normal(0.0, 10 * math.sqrt(kT / m), size=(s.num_particles, 3))
    if dim == 2:
        v[:, 2] = 0.0
    s.set("PART_VEL", v.ravel())
    s.step(1)
    cells = s.get("PART_CELL")
    vel = s.get("PART_VEL").reshape(-1, 3)[:, :dim]
    cut = _cut_mask(cells, p, s.get("SHIFT")[1])
    S, dof = 0.0, 0
    for c in np.unique(cells[~cut]):
        w = vel[cells == c]
        S += ((w - w.mean(0)) ** 2).sum()
        dof += dim * (w.shape[0] - 1)
    z = (S / (kT / m) - dof) / math.sqrt(2 * dof)
    assert dof > 5000
    assert abs(z) < 5, z


@pytest.mark.parametrize("dim", [2, 3])
def test_at_at_zero_temperature_every_particle_takes_the_cell_velocity(dim):
    """kT = 0: no random velocities, so each particle leaves with v_cm; in a
    wall-cut cell with n_c < ppc the ppc - n_c virtual particles at rest count
    in the mean (v_cm = sum v / ppc)."""
    a, b, p = _pair(dim, kT=0.0)
    rng = np.random.default_rng(5)
    v = rng.normal(0.0, 0.01, size=(a.num_particles, 3))
    if dim == 2:
        v[:, 2] = 0.0
    a.set("PART_VEL", v.ravel())
    b.set("PART_VEL", v.ravel())
    n_cut = 0
    for _ in range(4):
        a.step(1)
        b.step(1)
        cells = a.get("PART_CELL")
        va = a.get("PART_VEL").reshape(-1, 3)
        vb = b.get("PART_VEL").reshape(-1, 3)
        cut = _cut_mask(cells, p, a.get("SHIFT")[1])
        for c in np.unique(cells):
            mk = cells == c
            n = int(mk.sum())
            denom = p["ppc"] if (cut[mk][0] and n < p["ppc"]) else n
            n_cut += denom != n
            want = vb[mk].sum(0) / denom
            np.testing.assert_allclose(va[mk], np.broadcast_to(want, va[mk].shape), rtol=0, atol=1e-17)
        b.set("PART_VEL", va.ravel())
    assert n_cut > 0


def test_at_virtual_particles_in_wall_cells():
    """In a wall-cut cell with n < ppc the real particles' momentum changes by
    (n/ppc - 1) P_pre + (n/ppc)(P_virt - X_virt) + (1 - n/ppc) X_real, with
    P_virt, X_virt ~ N(0, (ppc - n) kT/m) and X_real ~ N(0, n kT/m) per
    component (Eq. 6 with the virtual particles as members of the cell), so
    its standardised value is N(0, 1)."""
    kT = 1e-3
    a, b, p = _pair(2, kT=kT, nx=24, ny=10)
    ppc = p["ppc"]
    zs = []
    for _ in range(12):
        a.step(1)
        b.step(1)
        cells = a.get("PART_CELL")
        va = a.get("PART_VEL").reshape(-1, 3)[:, :2]
        vb = b.get("PART_VEL").reshape(-1, 3)[:, :2]
        cut = _cut_mask(cells, p, a.get("SHIFT")[1])
        for c in np.unique(cells[cut]):
            mk = cells == c
            n = int(mk.sum())
            if n >= ppc:
                continue
            f = n / ppc
            P = vb[mk].sum(0)
            dP = va[mk].sum(0) - P
            var = f * f * 2 * (ppc - n) * kT + (1 - f) ** 2 * n * kT
            zs.extend((dP - (f - 1) * P) / math.sqrt(var))
        b.set("PART_VEL", a.get("PART_VEL"))
    zs = np.array(zs)
    assert zs.size > 200
    assert stats.kstest(zs, "norm").pvalue > 1e-4


def test_eq7_gives_table1_thermal_energies():
    """Table 1 lists, for nu_MPCD = nu_LB = 0.167, kT ~ 0.17 at a = 1 and
    kT ~ 0.3 at a = 1/2 (N = 60 ... 1000): Eq. 7 solved for kT gives them."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for run, a, N, nu, kT, tol in rows:
        got = T.at_kT_for_viscosity(float(nu), float(N), float(a))
        assert abs(got - float(kT)) <= float(tol), (run, a, N, got)
        kin, col = T.at_viscosity(float(N), got, float(a))
        assert abs(kin + col - float(nu)) < 1e-12


@pytest.mark.parametrize("over", [dict(collision=2), dict(collision=-1),
                                  dict(collision=1, resample_density=1)])
def test_collision_mode_is_validated(over):
    p = dict(lattice=9, nx=8, ny=6, nz=1, tau=1.0, ppc=4, coupling_width=0, feedback=0)
    p.update(over)
    with pytest.raises(ValueError):
        O.OracleSim(p)
