"""Pins of the oracle's MPCD part: streaming (Eq. 3), binning under the random
grid shift, SRD collision (Eq. 4), virtual wall particles, equilibrium noise
(Eq. 8).  Not GPU."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle as O
from tests import inputs

DEG = math.pi / 180.0


def toy(dim=2, **over):
    """4 x 4 (x 4) cell toy: no LB force, no coupling buffer."""
    if dim == 2:
        p = dict(lattice=9, nx=4, ny=6, nz=1, tau=1.0, force=(0, 0, 0), refine=1, ppc=4,
                 alpha=130 * DEG, kT=1e-4, coupling_width=0, feedback=0, seed=7)
    else:
        p = dict(lattice=19, nx=4, ny=6, nz=4, tau=1.0, force=(0, 0, 0), refine=1, ppc=3,
                 alpha=120 * DEG, kT=1e-4, coupling_width=0, feedback=0, seed=7)
    p.update(over)
    s = O.OracleSim(p)
    s.set_region(0, p["nx"])
    return s, p


def brute_force_cell(home, off, shift, W, Hy, Wz, dim):
    """Collision cell by interval membership on the shifted grid, exact rationals:
    the cell c along an axis is the one with c - s <= X < c + 1 - s."""
    idx = []
    for a in range(dim):
        X = Fraction(int(home[a])) + Fraction(float(off[a]))
        s = Fraction(float(shift[a]))
        c = None
        for cand in range(-1, (W, Hy, Wz)[a] + 2):
            if cand - s <= X < cand + 1 - s:
                c = cand
                break
        if a == 0:
            c %= W
        if a == 2:
            c %= Wz
        idx.append(c)
    if dim == 2:
        idx.append(0)
    return idx[0] + W * (idx[1] + (Hy + 1) * idx[2])


@pytest.mark.parametrize("dim,precision", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_binning_matches_brute_force(dim, precision):
    """Particles at rest (kT = 0, v = 0): every step's binning equals interval
    membership on the shifted grid, bit-exactly, in both precisions."""
    s, p = toy(dim, kT=0.0, precision=precision)
    n = s.num_particles
    s.set("PART_VEL", np.zeros(3 * n))
    home = s.get("PART_HOME").reshape(-1, 3)
    off = s.get("PART_POS").reshape(-1, 3)
    W, Hy, Wz = 4, 4, 4 if dim == 3 else 1
    for _ in range(6):
        s.step(1)
        assert np.array_equal(s.get("PART_HOME").reshape(-1, 3), home)
        sh = s.get("SHIFT")
        cells = s.get("PART_CELL")
        want = [brute_force_cell(home[k], off[k], sh, W, Hy, Wz, dim) for k in range(n)]
        assert np.array_equal(cells, want)
        assert np.array_equal(s.get("CELL_COUNT"), np.bincount(want, minlength=W * (Hy + 1) * Wz))


def test_binning_ties_go_to_upper_cell():
    """An offset exactly 1 - s sits on the shifted cell edge: it belongs to the
    upper cell.  One 2^-24 quantum below the edge it stays in the lower cell.
    One binary64 ulp below the edge the rounded sum off + s is 1.0, so the
    decision, taken in the storage precision, is the upper cell."""
    s, p = toy(2, kT=0.0)
    s.set("PART_VEL", np.zeros(3 * s.num_particles))
    s.step(1)
    sh = s.get("SHIFT")
    s2, _ = toy(2, kT=0.0)
    off = s2.get("PART_POS").reshape(-1, 3)
    off[0, 0] = 1.0 - sh[0]
    off[1, 1] = 1.0 - sh[1]
    off[2, 0] = 1.0 - sh[0] - 2.0 ** -24
    off[3, 0] = np.nextafter(1.0 - sh[0], 0.0)
    s2.set("PART_POS", off)
    s2.set("PART_VEL", np.zeros(3 * s2.num_particles))
    home = s2.get("PART_HOME").reshape(-1, 3)
    s2.step(1)
    cells = s2.get("PART_CELL")
    for k in range(3):
        assert cells[k] == brute_force_cell(home[k], off[k], sh, 4, 4, 1, 2)
    assert cells[0] % 4 == (home[0, 0] + 1) % 4
    assert cells[1] // 4 == home[1, 1] + 1
    assert cells[2] % 4 == home[2, 0]
    assert off[3, 0] + sh[0] == 1.0
    assert cells[3] % 4 == (home[3, 0] + 1) % 4


def _pair(dim, **over):
    """Two identical systems, one with the SRD angle and one with alpha = 0:
    the second's post-collision velocities are the pre-collision ones."""
    a, p = toy(dim, **over)
    b, _ = toy(dim, alpha=0.0, **over)
    return a, b, p


@pytest.mark.parametrize("dim", [2, 3])
def test_srd_conserves_cell_momentum_and_energy(dim):
    """Eq. 4 conserves each cell's momentum and kinetic energy (Sec. 2.2) in
    every cell not cut by a wall; v_cm is the cell mean."""
    a, b, p = _pair(dim)
    for _ in range(3):
        a.step(1)
        b.step(1)
        cells = a.get("PART_CELL")
        assert np.array_equal(cells, b.get("PART_CELL"))
        va = a.get("PART_VEL").reshape(-1, 3)
        vb = b.get("PART_VEL").reshape(-1, 3)
        ncx, ncy = 4, 5
        cy = (cells // ncx) % ncy
        cut = (cy == 0) | (cy == ncy - 1)
        vcm = a.get("CELL_VCM").reshape(-1, 3)
        for c in np.unique(cells[~cut]):
            m = cells == c
            np.testing.assert_allclose(va[m].sum(0), vb[m].sum(0), rtol=0, atol=1e-15)
            assert abs((va[m] ** 2).sum() - (vb[m] ** 2).sum()) < 1e-14 * (vb[m] ** 2).sum() + 1e-300
            np.testing.assert_allclose(vcm[c], vb[m].mean(0), rtol=0, atol=1e-16)
        # the two runs stay identical in position
        b.set("PART_VEL", va.ravel())


def test_srd_2d_rotation_angle_per_cell():
    """In 2D every particle of a cell turns by the same +alpha or -alpha about v_cm."""
    a, b, p = _pair(2)
    a.step(1)
    b.step(1)
    cells = a.get("PART_CELL")
    vcm = a.get("CELL_VCM").reshape(-1, 3)
    wa = a.get("PART_VEL").reshape(-1, 3)[:, :2] - vcm[cells, :2]
    wb = b.get("PART_VEL").reshape(-1, 3)[:, :2] - vcm[cells, :2]
    ang = np.arctan2(wb[:, 0] * wa[:, 1] - wb[:, 1] * wa[:, 0], (wb * wa).sum(1))
    np.testing.assert_allclose(np.linalg.norm(wa, axis=1), np.linalg.norm(wb, axis=1), atol=1e-15)
    signs = set()
    for c in np.unique(cells):
        m = (cells == c) & (np.linalg.norm(wb, axis=1) > 1e-12)
        if m.sum() == 0:
            continue
        sgn = np.sign(ang[m])
        assert np.all(sgn == sgn[0])
        np.testing.assert_allclose(np.abs(ang[m]), p["alpha"], atol=1e-9)
        signs.add(sgn[0])
    assert signs == {-1.0, 1.0}


def test_srd_mean_rotation_identities():
    """Average over +-alpha of R w is cos(alpha) w (2D); average over the six
    axes +-e_x, +-e_y, +-e_z of R(n, alpha) w is (1 + 2 cos alpha)/3 w (3D)."""
    rng = np.random.default_rng(2)
    for alpha in (130 * DEG, 120 * DEG, 0.3):
        for _ in range(10):
            v, vc = rng.normal(size=2), rng.normal(size=2)
            m = 0.5 * (O.srd_rotate_2d(v, vc, alpha, 1) + O.srd_rotate_2d(v, vc, alpha, -1))
            np.testing.assert_allclose(m - vc, math.cos(alpha) * (v - vc), atol=1e-14)
            v3, vc3 = rng.normal(size=3), rng.normal(size=3)
            axes = [s * e for e in np.eye(3) for s in (1, -1)]
            m3 = np.mean([O.srd_rotate_3d(v3, vc3, n, alpha) for n in axes], axis=0)
            np.testing.assert_allclose(m3 - vc3, (1 + 2 * math.cos(alpha)) / 3 * (v3 - vc3), atol=1e-14)
            # rotation about an axis parallel to w leaves w unchanged
            w = v3 - vc3
            np.testing.assert_allclose(O.srd_rotate_3d(v3, vc3, w / np.linalg.norm(w), alpha), v3, atol=1e-14)


def _stream_case(home, off, vel, force=(0.0, 0.0, 0.0), refine=1):
    """Place one moving particle among resting ones (kT = 0, alpha = 0)."""
    s, p = toy(2, kT=0.0, alpha=0.0, force=force, refine=refine)
    n = s.num_particles
    H = s.get("PART_HOME").reshape(-1, 3)
    X = s.get("PART_POS").reshape(-1, 3)
    V = np.zeros((n, 3))
    H[0, :2], X[0, :2], V[0, :2] = home, off, vel
    s.set("PART_HOME", H.ravel())
    s.set("PART_POS", X.ravel())
    s.set("PART_VEL", V.ravel())
    s.step(1)
    return (s.get("PART_HOME").reshape(-1, 3)[0], s.get("PART_POS").reshape(-1, 3)[0],
            s.get("PART_VEL").reshape(-1, 3)[0], s)


def _exact_path(X0, Y0, vx, vy, Hy, W):
    """Straight flight for one step; on reaching y = 0 or y = Hy the particle
    reverses its velocity and flies back for the rest of the step."""
    X0, Y0, vx, vy = map(Fraction, (X0, Y0, vx, vy))
    Y1 = Y0 + vy
    if 0 <= Y1 < Hy:
        return (X0 + vx) % W, Y1, vx, vy
    yw = 0 if Y1 < 0 else Hy
    ts = (yw - Y0) / vy
    Xh = X0 + vx * ts
    return (Xh - vx * (1 - ts)) % W, yw - vy * (1 - ts), -vx, -vy


@pytest.mark.parametrize("home,off,vel", [
    ((1, 0), (0.5, 0.1), (0.2, -0.3)),      # hits the bottom wall
    ((2, 3), (0.25, 0.875), (-0.125, 0.5)),  # hits the top wall (Hy = 4)
    ((3, 2), (0.9, 0.5), (0.3, 0.05)),       # periodic wrap in x
    ((0, 1), (0.05, 0.5), (-0.2, -0.75)),    # wraps in x, crosses a cell in y
])
def test_streaming_matches_exact_flight(home, off, vel):
    """Eq. 3 with bounce-back walls and periodic x against exact rational flight."""
    h, o, v, s = _stream_case(home, off, vel)
    Xe, Ye, vxe, vye = _exact_path(home[0] + off[0], home[1] + off[1], vel[0], vel[1], 4, 4)
    assert abs((h[0] + o[0]) - float(Xe)) < 1e-15 * 8
    assert abs((h[1] + o[1]) - float(Ye)) < 1e-15 * 8
    assert 0 <= o[0] < 1 and 0 <= o[1] < 1 and 0 <= h[1] < 4
    np.testing.assert_allclose(v[:2], [float(vxe), float(vye)], atol=1e-15)


def test_streaming_kick_then_drift_and_refinement():
    """The body force acts before the drift (v += g, r += v dt) and positions
    are in cell units, so a drift of v covers v r cells at refinement r."""
    g = (0.01, 0.0, 0.0)
    h, o, v, _ = _stream_case((1, 1), (0.25, 0.5), (0.1, 0.0), force=g, refine=2)
    np.testing.assert_allclose(v[0], 0.11, atol=1e-15)
    np.testing.assert_allclose(h[0] + o[0], 1.25 + 0.11 * 2, atol=1e-15)


def test_initial_state():
    """Exactly ppc particles per cell, Maxwellian velocities of variance kT/m."""
    cfg = inputs.small_2d(ppc=20, kT=2.5e-3)
    s = O.OracleSim(cfg["params"])
    s.set_region(*cfg["region"])
    home = s.get("PART_HOME").reshape(-1, 3)
    Wx = (cfg["region"][1] - cfg["region"][0]) * 2
    counts = np.bincount(home[:, 0] + Wx * home[:, 1])
    assert np.all(counts == 20)
    v = s.get("PART_VEL").reshape(-1, 3)
    z = v[:, :2].ravel() / math.sqrt(2.5e-3)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert np.all(v[:, 2] == 0)


def test_equilibrium_noise_of_cell_velocity():
    """Eq. 8 with N_s = 1: at rest the velocity of a cell of N particles has
    standard deviation sqrt(kT / (N m)) per component."""
    kT = 1e-3
    s, p = toy(2, kT=kT, ppc=10, nx=16, ny=18)
    s.step(3)
    cells = s.get("PART_CELL")
    cnt = s.get("CELL_COUNT")
    vcm = s.get("CELL_VCM").reshape(-1, 3)
    cy = (np.arange(cnt.size) // 16) % 17
    keep = (cnt > 0) & (cy > 0) & (cy < 16)
    z = vcm[keep, :2] * np.sqrt(cnt[keep, None] / kT)
    assert abs(z.std() - 1.0) < 0.06
    assert abs(z.mean()) < 0.1


def test_virtual_wall_particles():
    """A wall-cut cell with n_c < ppc receives ppc - n_c virtual particles whose
    total momentum is N(0, (ppc - n_c) m kT) per component."""
    kT = 1e-3
    zs = []
    a, b, p = _pair(2, kT=kT, nx=16, ny=10, ppc=6)
    for _ in range(10):
        b.step(1)
        cells = b.get("PART_CELL")
        cnt = b.get("CELL_COUNT")
        vcm = b.get("CELL_VCM").reshape(-1, 3)
        vb = b.get("PART_VEL").reshape(-1, 3)
        sy = b.get("SHIFT")[1]
        ncx, ncy = 16, 9
        for c in range(cnt.size):
            cy = (c // ncx) % ncy
            if cnt[c] == 0:
                continue
            if (cy == 0 or cy == ncy - 1) and sy > 0 and cnt[c] < 6:
                P = vcm[c, :2] * 6 - vb[cells == c, :2].sum(0)
                zs.extend(P / math.sqrt((6 - cnt[c]) * kT))
            else:
                np.testing.assert_allclose(vcm[c], vb[cells == c].mean(0), atol=1e-15)
    zs = np.array(zs)
    assert len(zs) > 100
    assert stats.kstest(zs, "norm").pvalue > 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_list_groups_particles_by_cell(dim):
    """CELL_LIST is the stable grouping of particle indices by collision cell:
    a permutation equal to a stable argsort of PART_CELL, with CELL_COUNT[c]
    entries for cell c."""
    cfg = inputs.small_2d() if dim == 2 else inputs.small_3d()
    s = O.OracleSim(cfg["params"])
    s.set_region(*cfg["region"])
    s.step(3)
    cells = s.get("PART_CELL")
    lst = s.get("CELL_LIST")
    assert np.array_equal(np.sort(lst), np.arange(len(cells)))
    assert np.array_equal(lst, np.argsort(cells, kind="stable"))
    cnt = s.get("CELL_COUNT")
    assert np.array_equal(np.bincount(cells[lst], minlength=len(cnt)), cnt)
    assert np.all(np.diff(cells[lst]) >= 0)
