"""x-slab decomposition on the GPU: the ranks of one channel emulated in one
process (run_local: every slab is its own handle, the host orders the halo
copies, nothing waits on anything) against the undivided channel's handle,
with the MPCD region whole in one slab or divided into pieces,
in FP64 (1e-12: only the order of the MPCD's binary64 atomics differs) and
FP32 (1e-5 of the populations' scale, the single-step tolerance); and the
halo calls' argument errors."""
import numpy as np
import pytest

from tests import inputs
from tests.test_slabs import _initial_pops

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_00304_gb300 as mod
    return mod


def _run_both(lb, p, region, world, halo, steps, P0=None):
    from paper_2004_00304_gb300 import slabs as S
    cuts = S.plan_slabs(p["nx"], world, S.column_costs(p, region), region, halo=halo)
    one = lb.Lbmpcd([p])
    one.set_region(0, *region)
    if P0 is not None:
        one.set("POPS", P0)
    one.step(steps)
    sl = [S.SlabChannel(p, cuts, r, region=region, halo=halo) for r in range(world)]
    if P0 is not None:
        for s in sl:
            s.set_global("POPS", P0)
    S.run_local(sl, steps)
    return one, sl, cuts


@pytest.mark.parametrize("world,halo,steps", [(2, 4, 23), (3, 2, 17), (1, 3, 10)])
def test_fp64_slabs_match_the_undivided_channel(lb, world, halo, steps):
    cfg = inputs.small_2d(feedback=1)
    p, region = cfg["params"], cfg["region"]
    P0 = _initial_pops(p)
    one, sl, cuts = _run_both(lb, p, region, world, halo, steps, P0)
    nx = p["nx"]
    R = one.get("POPS").reshape(9, 1, p["ny"], nx)
    scale = np.max(np.abs(R))
    for r, s in enumerate(sl):
        got = s.interior("POPS")
        want = R[..., np.arange(cuts[r], cuts[r + 1]) % nx]
        assert np.max(np.abs(got - want)) <= 1e-12 * scale, r
        if s.has_region:
            v1, v2 = one.get("PART_VEL"), s.sim.get("PART_VEL")
            assert np.max(np.abs(v1 - v2)) <= 1e-12 * max(1.0, np.max(np.abs(v1)))
    assert sum(s.has_region for s in sl) == 1
    one.close()
    for s in sl:
        s.close()


def _owned_particles(sl):
    """The union of the pieces' owned particles, ordered by particle id."""
    from paper_2004_00304_gb300 import slabs as S
    home, off, vel, pid = S._concat([s.particles_out() for s in sl])
    o = np.argsort(pid)
    return home[o], off[o], vel[o], pid[o]


@pytest.mark.parametrize("dim,world,halo,steps", [(2, 2, 2, 13), (2, 3, 2, 11), (2, 3, 4, 19), (3, 2, 2, 7)])
def test_fp64_divided_region_matches_the_undivided_channel(lb, dim, world, halo, steps):
    """The MPCD region cut between slabs: each slab's handle holds a region
    piece (its own cell columns plus ghost columns, particles handed over at
    every halo exchange, the imposition on its own columns only).  Against
    the undivided channel after steps that cross several LB exchanges (the
    particles change hands after every step): every interior population,
    and every particle's home cell (equal), offsets and velocities (the union
    of the pieces' own particles, by id) within 1e-12; each particle owned
    by exactly one piece."""
    from paper_2004_00304_gb300 import slabs as S
    cfg = inputs.small_2d(feedback=1) if dim == 2 else inputs.small_3d(feedback=1)
    p, region = cfg["params"], cfg["region"]
    q, nz = p["lattice"], p.get("nz", 1)
    P0 = _initial_pops(p)
    cuts = S.plan_slabs(p["nx"], world, S.column_costs(p, region), region, halo=halo, split_region=True,
                        cw=p["coupling_width"])
    one = lb.Lbmpcd([p])
    one.set_region(0, *region)
    one.set("POPS", P0)
    one.step(steps)
    sl = [S.SlabChannel(p, cuts, r, region=region, halo=halo) for r in range(world)]
    for s in sl:
        s.set_global("POPS", P0)
    npiece = sum(s.piece is not None for s in sl)
    assert npiece == world or (world > 1 and npiece >= 2), cuts
    S.run_local(sl, steps)
    nx = p["nx"]
    R = one.get("POPS").reshape(q, nz, p["ny"], nx)
    scale = np.max(np.abs(R))
    for r, s in enumerate(sl):
        got = s.interior("POPS")
        want = R[..., np.arange(cuts[r], cuts[r + 1]) % nx]
        assert np.max(np.abs(got - want)) <= 1e-12 * scale, r
    home, off, vel, pid = _owned_particles(sl)
    n = one.get("PART_ID").size
    assert pid.size == n and np.array_equal(pid, np.arange(n)), (pid.size, n)
    assert np.array_equal(home, one.get("PART_HOME").reshape(-1, 3))
    v1 = one.get("PART_VEL").reshape(-1, 3)
    assert np.max(np.abs(off - one.get("PART_POS").reshape(-1, 3))) <= 1e-12
    # velocities: every particle but those of the outer buffers, whose
    # post-collision velocity the next step's redraw replaces (their
    # collision cells at the region's periodic wrap hold ghost copies of the
    # far end's outer buffer, which a piece redraws from LB columns it does
    # not hold); their positions above are exact
    r_, wx = p["refine"], (region[1] - region[0]) * p["refine"]
    n_out = (p["coupling_width"] + 1) // 2
    inner = (home[:, 0] >= n_out * r_) & (home[:, 0] < wx - n_out * r_)
    assert inner.sum() > 0.5 * n
    assert np.max(np.abs(vel[inner] - v1[inner])) <= 1e-12 * max(1.0, np.max(np.abs(v1)))
    one.close()
    for s in sl:
        s.close()


def test_fp32_slabs_of_a_wide_channel(lb):
    """FP32, 512 x 64 channel with a 64-column MPCD region at r = 2, three
    slabs with 4 ghost columns, 40 steps from rest: every interior population
    within 1e-5 of the populations' scale of the undivided channel's."""
    p = dict(lattice=9, nx=512, ny=64, nz=1, tau=0.8, force=(1e-6, 0.0, 0.0), refine=2, ppc=10,
             alpha=130 * np.pi / 180, kT=1e-4, mass=1.0, coupling_width=2, precision=1, feedback=1,
             window=20, resample_density=0, seed=21)
    region = (224, 288)
    one, sl, cuts = _run_both(lb, p, region, 3, 4, 40)
    R = one.get("POPS").reshape(9, 1, 64, 512)
    for r, s in enumerate(sl):
        got = s.interior("POPS")
        want = R[..., np.arange(cuts[r], cuts[r + 1]) % 512]
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(R)), r
    one.close()
    for s in sl:
        s.close()


def test_column_calls_check_their_arguments(lb):
    import torch
    cfg = inputs.small_2d()
    g = lb.Lbmpcd([cfg["params"]])
    g.set("POPS", _initial_pops(cfg["params"]))                   # every column different
    nb = g.column_bytes(2)
    assert g.population_bytes() == 8
    buf = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    with pytest.raises(lb.LbmpcdError):
        g.get_columns(cfg["params"]["nx"] - 1, 2, buf)            # beyond the last column
    with pytest.raises(lb.LbmpcdError):
        g.get_columns(-1, 2, buf)
    with pytest.raises(ValueError):
        g.get_columns(0, 3, buf)                                  # buffer of the wrong size
    g.get_columns(3, 2, buf)
    host = np.zeros(nb, np.uint8)
    g.get_columns(3, 2, host)
    assert np.array_equal(host, buf.cpu().numpy())
    # round trip through another column pair of the lattice
    g.set_columns(10, 2, buf)
    P = g.get("POPS").reshape(9, 1, cfg["params"]["ny"], cfg["params"]["nx"])
    assert np.array_equal(P[..., 10:12], P[..., 3:5])
    assert not np.array_equal(P[..., 12:14], P[..., 3:5])
    g.close()
