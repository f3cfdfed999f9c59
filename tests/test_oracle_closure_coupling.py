"""Pins of the oracle's learned-closure coupling (feedback = 2): the strip
fields, their 8-frame history, the moving-average target, the patch layout
and the imposition from a network output.  Each is checked against something
computed independently of the oracle: particle counts and velocities read
back from the particle state, the closed form of the moving-average
recursion, and the moments of the imposed populations.  Not GPU."""
import math

import numpy as np
import pytest

import oracle as O
from tests import inputs

W = 16


def _cfg(**over):
    return inputs.small_2d(feedback=2, **over)


def _sim(cfg):
    s = O.OracleSim(cfg["params"])
    s.set_region(*cfg["region"])
    return s


def _geometry(cfg):
    p = cfg["params"]
    x0, x1 = cfg["region"]
    r = p["refine"]
    Wx, Hy = (x1 - x0) * r, (p["ny"] - 2) * r
    npy = -(-Hy // W)
    return Wx, Hy, npy


def _patch_rows(Hy, npy):
    """First fine row of each patch per side: 16 py, the last one Hy - 16."""
    return [Hy - W if py == npy - 1 else W * py for py in range(npy)]


def _strip_fields(cfg, home, vel):
    """Counts and mean velocities per strip cell from the particle state, laid
    out as (patch, row, xi) -- written here from the layout's description."""
    p = cfg["params"]
    Wx, Hy, npy = _geometry(cfg)
    sig = math.sqrt(p["kT"] / p["mass"])
    cnt = np.zeros((2, Hy, W))
    sv = np.zeros((2, Hy, W, 2))
    X, Y = home[:, 0], home[:, 1]
    for side in (0, 1):
        xi = X if side == 0 else Wx - 1 - X
        sel = xi < W
        np.add.at(cnt[side], (Y[sel], xi[sel]), 1.0)
        for a in (0, 1):
            np.add.at(sv[side, :, :, a], (Y[sel], xi[sel]), vel[sel, a])
    phi = np.zeros((2, Hy, W, 3))
    phi[..., 0] = cnt / p["ppc"] - 1.0
    with np.errstate(invalid="ignore", divide="ignore"):
        for a in (0, 1):
            m = np.where(cnt > 0, sv[..., a] / cnt / sig, 0.0)
            phi[..., 1 + a] = m
    phi[1, ..., 1] *= -1.0                       # the right strip is seen in a mirror
    rows = _patch_rows(Hy, npy)
    out = np.stack([phi[side, rows[py]:rows[py] + W] for side in (0, 1) for py in range(npy)])
    return out                                   # (P, 16, 16, 3)


def test_newest_frame_counts_match_particle_homes():
    """Channel block of the newest frame, density part: n / ppc - 1 with n the
    particles whose home cell is the strip cell (collisions do not move
    particles, so the post-step homes are the sampled ones)."""
    cfg = _cfg()
    s = _sim(cfg)
    for _ in range(3):
        s.step(1)
        x = s.get("CLOSURE_IN").reshape(-1, 16, 16, 8, 3)
        home = s.get("PART_HOME").reshape(-1, 3)
        vel = s.get("PART_VEL").reshape(-1, 3)
        ref = _strip_fields(cfg, home, vel)
        assert x.shape[0] == 2 * _geometry(cfg)[2] == s.closure_patches
        np.testing.assert_array_equal(x[:, :, :, 7, 0], ref[..., 0])


def test_newest_frame_velocities_with_zero_rotation():
    """With alpha = 0 the collision leaves every velocity unchanged (up to
    rounding), so the post-step velocities give the sampled cell means; the
    right strip's u_x carries the mirror sign."""
    cfg = _cfg(alpha=0.0)
    s = _sim(cfg)
    for _ in range(2):
        s.step(1)
    x = s.get("CLOSURE_IN").reshape(-1, 16, 16, 8, 3)
    ref = _strip_fields(cfg, s.get("PART_HOME").reshape(-1, 3), s.get("PART_VEL").reshape(-1, 3))
    assert np.max(np.abs(ref[..., 1:])) > 0.3      # thermal velocities, O(1) after scaling
    np.testing.assert_allclose(x[:, :, :, 7, 1:], ref[..., 1:], rtol=0, atol=1e-11)


def test_history_moves_one_slot_per_step_and_starts_at_zero():
    cfg = _cfg()
    s = _sim(cfg)
    s.step(1)
    x0 = s.get("CLOSURE_IN").reshape(-1, 16, 16, 8, 3)
    assert np.all(x0[:, :, :, :7] == 0.0)          # frames before step 0 are zeros
    prev = x0
    for _ in range(9):
        s.step(1)
        x = s.get("CLOSURE_IN").reshape(-1, 16, 16, 8, 3)
        np.testing.assert_array_equal(x[:, :, :, :7], prev[:, :, :, 1:])
        prev = x


def test_target_is_the_closed_form_of_the_moving_average():
    """e_K = (1-a)^K phi_0 + sum_{k=1..K} a (1-a)^(K-k) phi_k with a = 1/500,
    the solution of the recursion started at e_0 = phi_0."""
    cfg = _cfg()
    s = _sim(cfg)
    frames = []
    K = 12
    for _ in range(K + 1):
        s.step(1)
        frames.append(s.get("CLOSURE_IN").reshape(-1, 16, 16, 8, 3)[:, :, :, 7, :])
    a = 1.0 / 500.0
    ref = (1 - a) ** K * frames[0]
    for k in range(1, K + 1):
        ref = ref + a * (1 - a) ** (K - k) * frames[k]
    e = s.get("CLOSURE_TARGET").reshape(-1, 16, 16, 3)
    np.testing.assert_allclose(e, ref, rtol=0, atol=1e-13)


def _inner_nodes(cfg):
    p = cfg["params"]
    x0, x1 = cfg["region"]
    cw = p["coupling_width"]
    n_out, n_in = (cw + 1) // 2, cw // 2
    out = []
    for side in (0, 1):
        for col in range(n_in):
            x = x0 + n_out + col if side == 0 else x1 - 1 - n_out - col
            out.append((side, col, x))
    return out, n_out


def test_imposition_sets_the_moments_of_the_predicted_velocity():
    """With the output u_x = xi (column) and u_y = the fine row: once 8 frames
    exist (after step 7) the prediction is recorded, and from the next LB
    update on every inner node gets populations with density rho_LB and
    velocity sqrt(kT/m) times the mean over its r x r fine cells (u_x mirrored
    on the right).  Up to step 7 the populations equal those of a twin run
    that never imposes; at the first imposition (step 8) only the inner nodes
    differ from it."""
    cfg = _cfg()
    p = cfg["params"]
    Wx, Hy, npy = _geometry(cfg)
    r = p["refine"]
    sig = math.sqrt(p["kT"] / p["mass"])
    s = _sim(cfg)
    twin = _sim(cfg)
    P = s.closure_patches
    rows = _patch_rows(Hy, npy)
    y = np.zeros((P, 16, 16, 3))
    for pch in range(P):
        y[pch, :, :, 1] = np.arange(16)[None, :]
        y[pch, :, :, 2] = rows[pch % npy] + np.arange(16)[:, None]
    q, nx, ny = 9, p["nx"], p["ny"]
    c = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
    nodes, n_out = _inner_nodes(cfg)
    for n in range(10):
        s.step(1)
        twin.step(1)
        after = s.get("POPS").reshape(q, ny, nx)
        other = twin.get("POPS").reshape(q, ny, nx)
        if n <= 7:
            np.testing.assert_array_equal(after, other)
        else:
            rho = s.get("RHO").reshape(ny, nx)
            changed = np.zeros((ny, nx), bool)
            for side, col, x in nodes:
                xi_mean = (n_out + col) * r + (r - 1) / 2.0
                for yn in range(1, ny - 1):
                    row_mean = (yn - 1) * r + (r - 1) / 2.0
                    u = np.array([(1 if side == 0 else -1) * sig * xi_mean, sig * row_mean])
                    f = after[:, yn, x]
                    assert abs(f.sum() - rho[yn, x]) < 1e-14
                    np.testing.assert_allclose(f @ c, rho[yn, x] * u, rtol=1e-12, atol=1e-18)
                    changed[yn, x] = True
            if n == 8:
                np.testing.assert_array_equal(after[:, ~changed], other[:, ~changed])
        s.closure_impose(y)


@pytest.mark.parametrize("over,region", [(dict(), (20, 34)),           # 28 fine columns < 2 x 16
                                         (dict(ny=9), (20, 43)),       # 14 fine rows < 16
                                         (dict(kT=0.0), (20, 43))])
def test_closure_geometry_is_validated(over, region):
    cfg = _cfg(**over)
    s = O.OracleSim(cfg["params"])
    with pytest.raises(ValueError):
        s.set_region(*region)
