"""x-slab decomposition of one channel (host side, no GPU): the cut planner,
and two gloo ranks driving FP64 oracle slabs against the undivided oracle
channel (bit-exact: every interior column and every particle computes the
same arithmetic in the same order)."""
import os
import socket

import numpy as np
import pytest

from paper_2004_00304_gb300 import slabs as S
from tests import inputs


class OracleEngine:
    """The oracle behind the slab driver's engine methods (test side only)."""

    def __init__(self, params):
        import oracle
        self.p = dict(params)
        self.o = oracle.OracleSim(self.p)
        self.q, self.nz, self.ny, self.nx = int(self.p["lattice"]), int(self.p.get("nz", 1)), int(self.p["ny"]), \
            int(self.p["nx"])

    def set_region(self, replica, x0, x1):
        self.o.set_region(x0, x1)

    def step(self, k):
        self.o.step(k)

    def get(self, field, replica=0, out=None):
        return self.o.get(field)

    def set(self, field, value, replica=0):
        if field != "POPS" and not field.startswith("PART_"):
            raise ValueError("the oracle engine loads POPS and particles only")
        self.o.set(field, value)

    def column_bytes(self, n):
        return self.q * self.nz * self.ny * n * 8

    def _pops(self):
        return self.o.get("POPS").reshape(self.q, self.nz, self.ny, self.nx)

    def get_columns(self, x, n, out):
        out.numpy().view(np.float64)[:] = np.ascontiguousarray(self._pops()[..., x:x + n]).ravel()
        return out

    def set_columns(self, x, n, src):
        P = self._pops().copy()
        P[..., x:x + n] = src.numpy().view(np.float64).reshape(self.q, self.nz, self.ny, n)
        self.o.set("POPS", P)

    def close(self):
        pass


def _initial_pops(p, seed=5):
    """Equilibrium populations of a non-uniform velocity field (a sheared,
    x-modulated flow), so that the halo carries information."""
    import oracle
    q, nz, ny, nx = int(p["lattice"]), int(p.get("nz", 1)), int(p["ny"]), int(p["nx"])
    rng = np.random.default_rng(seed)
    P = np.zeros((q, nz, ny, nx))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                u = np.array([0.01 * np.sin(2 * np.pi * x / nx) + 0.002 * y / ny,
                              0.005 * np.cos(2 * np.pi * x / nx), 0.0]) + rng.normal(0, 1e-3, 3)
                if q == 9:
                    u[2] = 0.0
                P[:, z, y, x] = oracle.feq(q, 1.0 + 0.01 * rng.normal(), u)
    return P


def test_plan_keeps_region_whole_and_balances():
    p = dict(lattice=9, nx=2048, ny=512, refine=2, ppc=10, precision=1)
    region = (896, 1152)
    c = S.column_costs(p, region)
    for n in (1, 2, 3, 4, 8):
        cuts = S.plan_slabs(2048, n, c, region, halo=4, margin=2)
        assert len(cuts) == n + 1 and cuts[-1] - cuts[0] == 2048
        assert all(b - a >= 4 for a, b in zip(cuts[:-1], cuts[1:]))
        costs = [c[np.arange(a, b) % 2048].sum() for a, b in zip(cuts[:-1], cuts[1:])]
        block = c[894:1154].sum()
        holders = [r for r, (a, b) in enumerate(zip(cuts[:-1], cuts[1:]))
                   if (894 - a) % 2048 + 260 <= b - a]
        assert len(holders) == 1                         # the region and its margins in one slab
        # the largest slab costs no more than the region's block or an even share, plus one column
        assert max(costs) <= max(block, c.sum() / n) + c.max() + 1e-6
    # uniform cost, no region: equal widths
    assert S.plan_slabs(64, 4, halo=4) == [0, 16, 32, 48, 64]
    with pytest.raises(ValueError):
        S.plan_slabs(16, 5, halo=4)                      # slabs narrower than the halo
    with pytest.raises(ValueError):
        S.plan_slabs(64, 2, region=(1, 10), margin=2)    # margins leave the channel


def test_advance_beyond_halo_needs_an_exchange():
    cfg = inputs.small_2d()
    p = cfg["params"]
    cuts = S.plan_slabs(p["nx"], 2, region=cfg["region"], halo=3)
    sl = S.SlabChannel(p, cuts, 1, region=cfg["region"], halo=3, make_engine=OracleEngine, device="cpu")
    sl.advance(2)
    with pytest.raises(ValueError):
        sl.advance(2)
    sl.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, p, region, cuts, halo, steps, P0, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        sl = S.SlabChannel(p, cuts, rank, region=region, halo=halo, make_engine=OracleEngine, device="cpu")
        sl.set_global("POPS", P0)
        S.run_dist(sl, steps, S.DistExchanger())
        np.save(os.path.join(out_dir, f"pops{rank}.npy"), sl.interior("POPS"))
        if sl.has_region:
            np.save(os.path.join(out_dir, f"vel{rank}.npy"), sl.sim.get("PART_VEL"))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,halo,steps", [(2, 4, 23), (2, 1, 9), (3, 2, 14)])
def test_gloo_ranks_match_the_undivided_oracle(tmp_path, world, halo, steps):
    """world ranks (gloo, processes), each an oracle slab of the 70 x 22
    channel with its MPCD region on one rank; after `steps` steps (a number
    that is not a multiple of the halo, so that the last stretch ends between
    exchanges) every interior population and every particle velocity equals
    the undivided oracle run's bit for bit."""
    import oracle
    import torch.multiprocessing as mp
    oracle.lib()                                         # built before the ranks start
    cfg = inputs.small_2d(feedback=1)
    p, region = cfg["params"], cfg["region"]
    P0 = _initial_pops(p)
    cuts = S.plan_slabs(p["nx"], world, S.column_costs(p, region), region, halo=halo)
    mp.spawn(_rank_main, args=(world, _free_port(), p, region, cuts, halo, steps, P0, str(tmp_path)),
             nprocs=world, join=True)
    ref = oracle.OracleSim(p)
    ref.set_region(*region)
    ref.set("POPS", P0)
    ref.step(steps)
    R = ref.get("POPS").reshape(9, 1, p["ny"], p["nx"])
    nx = p["nx"]
    for r in range(world):
        got = np.load(tmp_path / f"pops{r}.npy")
        cols = np.arange(cuts[r], cuts[r + 1]) % nx
        assert np.array_equal(got, R[..., cols]), r
    holders = [r for r in range(world) if (tmp_path / f"vel{r}.npy").exists()]
    assert len(holders) == 1
    assert np.array_equal(np.load(tmp_path / f"vel{holders[0]}.npy"), ref.get("PART_VEL"))


class PieceEngine:
    """A stand-in engine for the particle hand-over of a divided region (test
    side, no method physics): the whole region is seeded with one particle
    per cell, id = cell index, and every step moves every particle one cell
    to the right (periodic in the region), so that particles cross the cuts
    and change owner; the LB columns are zeros."""

    def __init__(self, params):
        self.p = dict(params)
        self.q, self.nz, self.ny = int(self.p["lattice"]), int(self.p.get("nz", 1)), int(self.p["ny"])
        self.r = int(self.p.get("refine", 1))

    def set_region_piece(self, replica, x0, x1, own, keep):
        self.wx, self.hy = (x1 - x0) * self.r, (self.ny - 2) * self.r
        self.own, self.keep = own, keep
        home, off, vel, pid = seeded(self.wx, self.hy)
        m = ((home[:, 0] - keep[0]) % self.wx) < (keep[1] - keep[0])
        self.set_particles(0, home[m], off[m], vel[m], pid[m])

    def set_particles(self, replica, home, off, vel, pid):
        self.home, self.off, self.vel, self.pid = (np.array(a) for a in (home, off, vel, pid))

    def get(self, field, replica=0, out=None):
        return {"PART_HOME": self.home, "PART_POS": self.off, "PART_VEL": self.vel, "PART_ID": self.pid}[field]

    def step(self, k):
        self.home = self.home.copy()
        self.home[:, 0] = (self.home[:, 0] + k) % self.wx

    def column_bytes(self, n):
        return self.q * self.nz * self.ny * n * 8

    def get_columns(self, x, n, out):
        return out

    def set_columns(self, x, n, src):
        pass

    def close(self):
        pass


def seeded(wx, hy):
    X, Y = np.meshgrid(np.arange(wx), np.arange(hy))
    home = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size, int)], 1).astype(np.int32)
    pid = (home[:, 0] + wx * home[:, 1]).astype(np.int32)
    off = np.full((pid.size, 3), 0.25)
    vel = np.stack([pid * 1e-3, -pid * 1e-3, np.zeros(pid.size)], 1)
    return home, off, vel, pid


def _divided(world, halo):
    cfg = inputs.small_2d(feedback=1)
    p, region = cfg["params"], cfg["region"]
    cuts = S.plan_slabs(p["nx"], world, S.column_costs(p, region), region, halo=halo, split_region=True,
                        cw=p["coupling_width"])
    return p, region, cuts


def test_plan_may_cut_the_region_away_from_its_buffers():
    p, region, cuts = _divided(3, 2)
    x0, x1 = region
    assert len(cuts) == 4 and cuts[-1] - cuts[0] == p["nx"]
    inner = [c % p["nx"] for c in cuts[1:-1]]
    assert any(x0 < c < x1 for c in inner)                 # the region is divided
    for c in cuts[:-1]:                                   # no cut within halo of a coupling buffer
        c %= p["nx"]
        assert not (x0 - 2 < c < x0 + 2 + 2) and not (x1 - 2 - 2 < c < x1 + 2)
    with pytest.raises(ValueError):
        S.plan_slabs(p["nx"], 2, region=(1, 30), halo=4, split_region=True)


@pytest.mark.parametrize("world,halo,steps", [(2, 2, 9), (3, 2, 11), (3, 4, 13)])
def test_pieces_hand_particles_over(world, halo, steps):
    """Slabs emulated in one process with a divided region: after steps that
    cross several LB exchanges, the pieces' owned particles are exactly the
    whole region's particles, each owned once, and every piece holds exactly
    the particles of its kept columns (modulo the region's width)."""
    p, region, cuts = _divided(world, halo)
    sl = [S.SlabChannel(p, cuts, r, region=region, halo=halo, make_engine=PieceEngine, device="cpu")
          for r in range(world)]
    pieces = [s for s in sl if s.piece is not None]
    assert len(pieces) >= 2
    S.run_local(sl, steps)
    wx = pieces[0].piece["wx"]
    home, off, vel, pid = seeded(wx, (p["ny"] - 2) * p["refine"])
    home = home.copy()
    home[:, 0] = (home[:, 0] + steps) % wx
    got = S._concat([s.particles_out() for s in sl])
    o = np.argsort(got[3])
    assert np.array_equal(got[3][o], np.sort(pid))
    assert np.array_equal(got[0][o], home[np.argsort(pid)])
    assert np.array_equal(got[2][o], vel[np.argsort(pid)])
    for s in pieces:                                      # handed over after every step: the kept columns
        k0, k1 = s.piece["keep"]
        want = np.sort(pid[((home[:, 0] - k0) % wx) < (k1 - k0)])
        assert np.array_equal(np.sort(s.sim.pid), want)


def _piece_rank_main(rank, world, port, p, region, cuts, halo, steps, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        sl = S.SlabChannel(p, cuts, rank, region=region, halo=halo, make_engine=PieceEngine, device="cpu")
        S.run_dist(sl, steps, S.DistExchanger())
        own = sl.particles_out()
        if own is not None:
            np.save(os.path.join(out_dir, f"home{rank}.npy"), own[0])
            np.save(os.path.join(out_dir, f"pid{rank}.npy"), own[3])
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,halo,steps", [(2, 2, 9), (3, 2, 11)])
def test_gloo_pieces_hand_particles_over(tmp_path, world, halo, steps):
    """The same hand-over between gloo ranks (one all-gather of the owned
    particles per step): their owned sets partition the region's particles,
    at the positions the undivided motion gives."""
    import torch.multiprocessing as mp
    p, region, cuts = _divided(world, halo)
    mp.spawn(_piece_rank_main, args=(world, _free_port(), p, region, cuts, halo, steps, str(tmp_path)),
             nprocs=world, join=True)
    wx = (region[1] - region[0]) * p["refine"]
    home, off, vel, pid = seeded(wx, (p["ny"] - 2) * p["refine"])
    home[:, 0] = (home[:, 0] + steps) % wx
    holders = [r for r in range(world) if (tmp_path / f"pid{r}.npy").exists()]
    assert len(holders) >= 2
    pids = np.concatenate([np.load(tmp_path / f"pid{r}.npy") for r in holders])
    homes = np.concatenate([np.load(tmp_path / f"home{r}.npy") for r in holders])
    o = np.argsort(pids)
    assert np.array_equal(pids[o], np.sort(pid))
    assert np.array_equal(homes[o], home[np.argsort(pid)])
