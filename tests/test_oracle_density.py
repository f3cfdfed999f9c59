"""Pins of the oracle's density resampling of the outer buffer
(resample_density = 1): particle counts drawn from the local LB density by
unbiased stochastic rounding, fresh uniform positions, Maxwellian velocities
about the interpolated LB velocity, the interior untouched.  Not GPU."""
import numpy as np
import pytest
from scipy import stats

import oracle as O
from tests import inputs


def _cfg(**over):
    base = dict(resample_density=1, feedback=0, force=(0.0, 0.0, 0.0))
    base.update(over)
    return inputs.small_2d(**base)


def _uniform_density(s, p, rho):
    """LB at rest with density rho everywhere (wall rows included)."""
    feq = O.feq(9, rho, [0.0, 0.0, 0.0])
    s.set("POPS", np.repeat(feq[:, None], p["ny"] * p["nx"], axis=1).ravel())


def _outer_mask(cfg, home):
    p = cfg["params"]
    x0, x1 = cfg["region"]
    n_out = (p["coupling_width"] + 1) // 2
    col = x0 + home[:, 0] // p["refine"]
    return (col < x0 + n_out) | (col >= x1 - n_out)


def test_counts_follow_the_density_by_stochastic_rounding():
    """At rest (kT = 0, g = 0) with uniform density 1.05 nothing moves: each
    outer cell holds floor(ppc 1.05) particles or one more, interior cells keep
    their ppc particles, and over all outer cells the mean count is ppc rho
    within a binomial 4-sigma band (the rounding is unbiased)."""
    cfg = _cfg(kT=0.0)
    p = cfg["params"]
    s = O.OracleSim(p)
    s.set_region(*cfg["region"])
    _uniform_density(s, p, 1.05)
    s.step(1)
    home = s.get("PART_HOME").reshape(-1, 3)
    x0, x1 = cfg["region"]
    Wx, Hy = (x1 - x0) * p["refine"], (p["ny"] - 2) * p["refine"]
    counts = np.bincount(home[:, 0] + Wx * home[:, 1], minlength=Wx * Hy)
    cols = np.arange(Wx * Hy) % Wx
    outer = _outer_mask(cfg, np.stack([cols, np.zeros_like(cols)], 1))
    rho = s.get("RHO").reshape(p["ny"], p["nx"])
    assert np.allclose(rho[1:-1], 1.05, atol=1e-12)
    x = p["ppc"] * 1.05
    assert np.all((counts[outer] == np.floor(x)) | (counts[outer] == np.floor(x) + 1))
    assert np.all(counts[~outer] == p["ppc"])
    frac = x - np.floor(x)
    m = counts[outer].size
    assert abs(counts[outer].mean() - x) < 4 * np.sqrt(frac * (1 - frac) / m)


def test_spawned_positions_and_velocities():
    """With alpha = 0 and g = 0 (collision and kick leave velocities as they
    are) the particles created in one step -- appended after the survivors --
    have offsets uniform in [0,1) and velocities N(u_LB, kT/m) per component;
    survivors are the previous interior particles, unchanged in number."""
    cfg = _cfg(alpha=0.0)
    p = cfg["params"]
    s = O.OracleSim(p)
    s.set_region(*cfg["region"])
    home0 = s.get("PART_HOME").reshape(-1, 3)
    n_interior = int((~_outer_mask(cfg, home0)).sum())
    s.step(1)
    n = s.num_particles
    assert n > n_interior
    vel = s.get("PART_VEL").reshape(-1, 3)[n_interior:]
    off = s.get("PART_POS").reshape(-1, 3)[n_interior:]
    sig = np.sqrt(p["kT"] / p["mass"])
    for a in (0, 1):
        assert stats.kstest(off[:, a], "uniform").pvalue > 1e-3
        assert stats.kstest(vel[:, a] / sig, "norm").pvalue > 1e-3   # LB at rest: u_fine = 0
    assert np.all(off[:, 2] == 0.0) and np.all(vel[:, 2] == 0.0)


def test_particle_count_bookkeeping_over_steps():
    """Each step removes the outer-buffer particles and adds the drawn counts:
    the total equals the interior survivors plus the new particles, and every
    particle stays inside the region with offsets in [0,1)."""
    cfg = _cfg(force=(2e-5, 0.0, 0.0))
    p = cfg["params"]
    s = O.OracleSim(p)
    s.set_region(*cfg["region"])
    x0, x1 = cfg["region"]
    Wx, Hy = (x1 - x0) * p["refine"], (p["ny"] - 2) * p["refine"]
    for _ in range(5):
        home = s.get("PART_HOME").reshape(-1, 3)
        s.step(1)
        n = s.num_particles
        h = s.get("PART_HOME").reshape(-1, 3)
        o = s.get("PART_POS").reshape(-1, 3)
        assert h.shape[0] == n
        assert np.all((h[:, 0] >= 0) & (h[:, 0] < Wx) & (h[:, 1] >= 0) & (h[:, 1] < Hy))
        assert np.all((o[:, :2] >= 0.0) & (o[:, :2] < 1.0))
    # close to ppc per cell on average (density near 1)
    assert abs(n / (Wx * Hy) - p["ppc"]) < 0.5


def test_density_mode_is_validated():
    p = inputs.small_2d(resample_density=2)["params"]
    with pytest.raises(ValueError):
        O.OracleSim(p)
