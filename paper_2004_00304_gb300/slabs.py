"""x-slab decomposition of one channel over ranks (host side).

The paper runs one domain.  A channel too large or too slow for one GPU is cut
into slabs of whole LB columns [X_r, X_r+1), one per rank.  Rank r's handle
holds its slab plus `halo` ghost columns on each side: local column = (global
column - X_r) mod nx + halo, local lattice nx_r = (X_r+1 - X_r) + 2 halo,
periodic in x like the whole channel.  The pull update (Sec. 2.1) reads only a node's
nearest neighbours, so the wrong values a ghost column pulls from beyond its
own edge move inwards by one column per step: after an exchange that refreshes
all `halo` ghost columns from the neighbours' interior columns, `halo` steps
leave every interior column exactly as the undivided channel computes it.  The
driver therefore takes `halo` steps, exchanges `halo` columns per cut in each
direction (raw population storage, lbmpcd_get_columns / lbmpcd_set_columns),
and repeats: one exchange every `halo` steps instead of one per step.

The MPCD region is either kept whole or divided.  Kept whole (the default),
plan_slabs places every cut outside the region and its `margin` LB columns on
either side (room for the buffers' interpolation stencils), so that the rank
that holds the region runs the coupled step of the undivided channel on it,
particles, cell table and coupling buffers included; the strong-scaling gain
is then bounded by total cost / region cost (1.45 for the 2048 x 512 channel
with its 256-column region).  Divided (split_region=True), cuts may fall
inside the region, but not within `halo` columns of its coupling buffers
(the imposition of a buffer node must not reach another slab's ghost
columns): each slab holding region columns runs a region piece
(lbmpcd_set_region_piece) that owns the region's cell columns inside the slab
and keeps, besides its own particles, those of `ghost` LB columns on each
side (modulo the region's periodic width).  Its cells, table and coupling
are those of the whole region, the imposition is applied on its own columns
only.  After every step each piece hands the particles it owned before the
step (in their new state, after the collision of the step) to every piece,
and each piece keeps those of its columns (lbmpcd_set_particles), ghosts
refreshed from their owners: the owner computed the step from complete
cells (a particle's collision cell is its home cell or the next one, and it
moves less than a cell per step, so one step of ghost columns suffices) and
from its own LB columns.  The hand-over is every step, not every `halo`
steps, because a particle may cross the region's periodic wrap from one
outer buffer into the other, where its next redraw needs the LB velocity of
the far end, which only the piece holding that end has.

Exchanges: DistExchanger (torch.distributed point-to-point, gloo on host
tensors or NCCL on device tensors) between processes, one rank each;
run_local() steps several slabs held by one process in lock step and hands
the halos over in memory (the form the tests use on one GPU: nothing waits on
anything, the host orders every copy).
"""
from __future__ import annotations

import numpy as np


def column_costs(params: dict, region=None) -> np.ndarray:
    """Per-column cost of the coupled step: algorithmic bytes of the LB update
    (2 q s per node, s = storage bytes) plus, in the MPCD region's columns,
    the particles' state (one read and one write, 2 (4 + 4 D) B per particle
    in binary32: position offset and velocity) and the collision cells'
    table (24 B per cell)."""
    q = int(params.get("lattice", 9))
    ny, nz = int(params["ny"]), int(params.get("nz", 1))
    prec = int(params.get("precision", 1))
    s = {0: 8, 1: 4, 2: 2}[prec]
    cost = np.full(int(params["nx"]), 2.0 * q * s * ny * nz)
    if region is not None:
        d = 3 if q == 19 else 2
        r, ppc = int(params.get("refine", 1)), int(params.get("ppc", 10))
        cells = r * (ny - 2) * r * (nz * r if d == 3 else 1)     # fine cells per LB column
        per_part = 2 * (4 + 4 * d) * (2 if prec == 0 else 1)
        cost[region[0]:region[1]] += cells * (ppc * per_part + 24)
    return cost


def plan_slabs(nx: int, nranks: int, cost=None, region=None, halo: int = 4, margin: int = 2,
               split_region: bool = False, cw: int = 2) -> list:
    """Cut positions X_0 < X_1 < ... < X_nranks = X_0 + nx of contiguous slabs
    of the periodic channel (slab r = columns [X_r, X_r+1) mod nx) that
    minimise the largest slab cost (`cost` per column, default uniform),
    every slab at least `halo` columns wide, the columns [x0 - margin,
    x1 + margin) of `region` = (x0, x1) inside one slab (the first: X_0 =
    x0 - margin, so that the rest of the channel, wrapping through x = 0, is
    one stretch).  ValueError when no such cut exists."""
    if nranks < 1:
        raise ValueError("need at least one rank")
    c = np.ones(nx) if cost is None else np.asarray(cost, dtype=np.float64)
    if c.size != nx:
        raise ValueError("one cost per column")
    shift = 0
    items = []                                        # (first column, width, cost), from column `shift` on
    if region is not None and split_region:
        # the region may be cut, but not within `halo` columns of its coupling
        # buffers: [x0 - halo, x0 + cw + halo) and [x1 - cw - halo, x1 + halo)
        # are each indivisible
        x0, x1 = region
        a0, a1, b0, b1 = x0 - halo, x0 + cw + halo, x1 - cw - halo, x1 + halo
        if a0 < 0 or b1 > nx or a1 > b0:
            raise ValueError("region, its buffers and their halos must lie inside the channel, the two ends apart")
        shift = a0
        items.append((a0, a1 - a0, float(c[a0:a1].sum())))
        items += [(x, 1, float(c[x])) for x in range(a1, b0)]
        items.append((b0, b1 - b0, float(c[b0:b1].sum())))
        items += [(x, 1, float(c[x % nx])) for x in range(b1, a0 + nx)]
    elif region is not None:
        blo, bhi = region[0] - margin, region[1] + margin
        if blo < 0 or bhi > nx or region[1] <= region[0]:
            raise ValueError("region and its margins must lie inside the channel")
        shift = blo
        items.append((blo, bhi - blo, float(c[blo:bhi].sum())))   # the region's block, indivisible
        items += [(x, 1, float(c[x % nx])) for x in range(bhi, blo + nx)]
    else:
        items = [(x, 1, float(c[x])) for x in range(nx)]

    def greedy(cap):
        groups, cur = [], []
        for it in items:
            w = sum(i[1] for i in cur)
            if cur and sum(i[2] for i in cur) + it[2] > cap and w >= halo:
                groups.append(cur)
                cur = []
            cur.append(it)
        groups.append(cur)
        return groups

    def fits(groups, cap):
        return len(groups) <= nranks and all(sum(i[1] for i in g) >= halo for g in groups) and \
            all(sum(i[2] for i in g) <= cap or len(g) == 1 for g in groups)

    total = float(c.sum())
    lo = max(total / nranks, max(i[2] for i in items))
    hi = total
    if not fits(greedy(hi), hi):
        raise ValueError("no cut with slabs of at least `halo` columns")
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if fits(greedy(mid), mid):
            hi = mid
        else:
            lo = mid
    groups = greedy(hi)
    # fewer groups than ranks: split the costliest group that can be split
    while len(groups) < nranks:
        best = None
        for gi, g in enumerate(groups):
            for k in range(1, len(g)):
                a, b = g[:k], g[k:]
                if sum(i[1] for i in a) >= halo and sum(i[1] for i in b) >= halo:
                    key = (sum(i[2] for i in g), -max(sum(i[2] for i in a), sum(i[2] for i in b)))
                    if best is None or key > best[0]:
                        best = (key, gi, k)
        if best is None:
            raise ValueError("too many ranks for this channel and halo")
        _, gi, k = best
        g = groups.pop(gi)
        groups[gi:gi] = [g[:k], g[k:]]
    return [g[0][0] for g in groups] + [shift + nx]


class SlabChannel:
    """One rank's slab of a channel: its engine (an Lbmpcd handle unless
    `make_engine` builds another with the same methods) on the local lattice,
    and the halo bookkeeping.  params: the whole channel's parameters; cuts:
    plan_slabs' output; region: the whole channel's MPCD region (x0, x1) or
    None (set on the rank whose slab holds it)."""

    def __init__(self, params: dict, cuts, rank: int, region=None, halo: int = 4, make_engine=None,
                 device: str = "cuda", stream=None, ghost=None):
        self.rank, self.world, self.halo = int(rank), len(cuts) - 1, int(halo)
        self.X0, self.X1 = int(cuts[rank]), int(cuts[rank + 1])
        self.w = self.X1 - self.X0
        if self.w < self.halo:
            raise ValueError("slab narrower than its halo")
        self.global_params = dict(params)
        self.local_params = dict(params, nx=self.w + 2 * self.halo)
        if make_engine is None:
            from . import Lbmpcd
            self.sim = Lbmpcd([self.local_params], stream=stream)
        else:
            self.sim = make_engine(self.local_params)
        nx = int(params["nx"])
        rel = None if region is None else (region[0] - self.X0) % nx      # region start inside the slab
        self.has_region = rel is not None and rel + (region[1] - region[0]) <= self.w
        self.piece = None
        self._own_ids = None
        if self.has_region:
            self.sim.set_region(0, rel + self.halo, rel + (region[1] - region[0]) + self.halo)
        elif region is not None:
            self._set_piece(region, rel, ghost)
        self.since = 0                                 # steps since the ghost columns were exact
        self.device = device
        nb = self.sim.column_bytes(self.halo)
        import torch
        self._buf = {k: torch.empty(nb, dtype=torch.uint8, device=device)
                     for k in ("send_left", "send_right", "recv_left", "recv_right")}

    def _set_piece(self, region, rel, ghost) -> None:
        """This slab holds part of a region that plan_slabs(split_region=True)
        divided: a region piece owning the region's columns inside the slab,
        keeping also the particles of `ghost` LB columns (default: enough for
        `halo` steps, 2 halo + 1 cells) on each side, modulo the region's
        periodic width."""
        x0g, x1g = region
        wlb = x1g - x0g
        if rel >= self.w + self.halo:                  # the region lies left of the slab's start
            rel -= int(self.global_params["nx"])
        lo = max(self.halo, rel + self.halo)
        hi = min(self.halo + self.w, rel + self.halo + wlb)
        if lo >= hi:
            return                                     # no region column in this slab
        r = int(self.global_params.get("refine", 1))
        g = int(ghost) if ghost is not None else -(-(2 * self.halo + 1) // r)
        c0, c1 = (lo - rel - self.halo) * r, (hi - rel - self.halo) * r     # owned region cell columns
        wx = wlb * r
        k0, k1 = c0 - g * r, c1 + g * r
        if k1 - k0 > wx:
            k0, k1 = 0, wx
        self.sim.set_region_piece(0, rel + self.halo, rel + self.halo + wlb, (lo, hi), (k0, k1))
        self.piece = dict(own=(c0, c1), keep=(k0, k1), wx=wx)
        home = self.sim.get("PART_HOME").reshape(-1, 3)
        pid = self.sim.get("PART_ID").reshape(-1)
        self._own_ids = pid[(home[:, 0] >= c0) & (home[:, 0] < c1)]   # owned before the first step

    def particles_out(self):
        """The particles this piece owned at the last hand-over (home cell
        column in its own columns then), in their current state after the
        collision of the last step, as (home [n][3], offsets [n][3],
        velocities [n][3], ids [n]).  The piece that owned a particle at the
        last hand-over computed its step from complete cells and from its own
        LB columns, also when the particle crossed into another piece's
        columns or, through the region's periodic wrap, into the far outer
        buffer during the step."""
        if self.piece is None:
            return None
        home = self.sim.get("PART_HOME").reshape(-1, 3)
        off = self.sim.get("PART_POS").reshape(-1, 3)
        vel = self.sim.get("PART_VEL").reshape(-1, 3)
        pid = self.sim.get("PART_ID").reshape(-1)
        m = np.isin(pid, self._own_ids)
        return home[m], off[m], vel[m], pid[m]

    def particles_in(self, owned) -> None:
        """Replace this piece's particles by those of `owned` (the owned sets
        of every piece, concatenated) in its kept columns, ordered by home
        cell; the ones in its own columns are its owned set until the next
        hand-over."""
        if self.piece is None:
            return
        home, off, vel, pid = owned
        k0, k1 = self.piece["keep"]
        c0, c1 = self.piece["own"]
        wx = self.piece["wx"]
        m = ((home[:, 0] - k0) % wx) < (k1 - k0)
        key = home[m, 0] + wx * (home[m, 1] + 1048576 * home[m, 2])
        o = np.argsort(key, kind="stable")
        self.sim.set_particles(0, home[m][o], off[m][o], vel[m][o], pid[m][o])
        self._own_ids = pid[(home[:, 0] >= c0) & (home[:, 0] < c1)]

    def global_columns(self) -> np.ndarray:
        """Global columns of the local lattice, ghosts included (mod nx)."""
        nx = int(self.global_params["nx"])
        return (np.arange(self.X0 - self.halo, self.X1 + self.halo)) % nx

    def set_global(self, field: str, value) -> None:
        """Load a whole-channel POPS [q][nz][ny][nx] or U [3][nz][ny][nx] (or
        the particles of the region's slab: PART_* fields pass through); the
        ghost columns get the neighbours' values, so the slab is exact at once."""
        if field in ("POPS", "U"):
            a = np.asarray(value, dtype=np.float64)
            p = self.global_params
            a = a.reshape(-1, int(p.get("nz", 1)), int(p["ny"]), int(p["nx"]))
            self.sim.set(field, np.ascontiguousarray(a[..., self.global_columns()]))
        else:
            self.sim.set(field, value)
        self.since = 0

    def advance(self, k: int) -> None:
        if self.since + k > self.halo:
            raise ValueError("more steps than the ghost columns cover: exchange first")
        self.sim.step(k)
        self.since += k

    def halo_out(self):
        """(to the left neighbour, to the right neighbour): the first and the
        last `halo` interior columns."""
        h = self.halo
        self.sim.get_columns(h, h, self._buf["send_left"])
        self.sim.get_columns(self.w, h, self._buf["send_right"])
        return self._buf["send_left"], self._buf["send_right"]

    def halo_in(self, from_left, from_right) -> None:
        """Ghost columns from the left neighbour's last and the right
        neighbour's first `halo` interior columns."""
        h = self.halo
        self.sim.set_columns(0, h, from_left)
        self.sim.set_columns(self.w + h, h, from_right)
        self.since = 0

    def interior(self, field: str) -> np.ndarray:
        """The slab's own columns of RHO / U / POPS, shape [comp][nz][ny][w]
        (global columns X_r .. X_r+1 - 1, mod nx)."""
        p = self.global_params
        a = self.sim.get(field).reshape(-1, int(p.get("nz", 1)), int(p["ny"]), self.w + 2 * self.halo)
        return a[..., self.halo:self.halo + self.w]

    def close(self) -> None:
        self.sim.close()


class DistExchanger:
    """Halo hand-over between ranks of a torch.distributed group (one slab
    per process): point-to-point sends to both ring neighbours and receives
    from both, posted as one batch; the leftward message carries tag 0 and
    the rightward tag 1, and the posting order (send left, send right, receive
    from the right, receive from the left) matches the two messages between
    the same pair of ranks when there are only two (NCCL matches by order)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def gather(self, obj):
        """Every rank's `obj` (host data), in rank order."""
        if self.world == 1:
            return [obj]
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out

    def exchange(self, send_left, send_right, recv_left, recv_right):
        if self.world == 1:
            recv_left.copy_(send_right)
            recv_right.copy_(send_left)
            return recv_left, recv_right
        d = self.dist
        left, right = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        gl = d.get_global_rank(self.group, left) if self.group is not None else left
        gr = d.get_global_rank(self.group, right) if self.group is not None else right
        ops = [d.P2POp(d.isend, send_left, gl, self.group, 0),
               d.P2POp(d.isend, send_right, gr, self.group, 1),
               d.P2POp(d.irecv, recv_right, gr, self.group, 0),
               d.P2POp(d.irecv, recv_left, gl, self.group, 1)]
        for w in d.batch_isend_irecv(ops):
            w.wait()
        return recv_left, recv_right


def _concat(parts):
    """The owned particle sets of all pieces (None for slabs without one) as
    one set."""
    parts = [p for p in parts if p is not None]
    if not parts:
        return None
    return tuple(np.concatenate([p[i] for p in parts]) for i in range(4))


def run_dist(slab: SlabChannel, steps: int, ex: DistExchanger) -> None:
    """`steps` steps of this rank's slab, exchanging with the other ranks (all
    ranks call it with the same `steps`): the LB ghost columns every `halo`
    steps; with a divided region also the particles after every step (one
    all-gather of the pieces' owned particles, each piece keeping those of
    its kept columns).  A particle may cross the region's periodic wrap from
    one outer buffer into the other, where the next step redraws it from the
    LB columns of the far end, which only the piece there holds: so the
    particles change hands every step."""
    pieces = ex.gather(slab.piece is not None)
    divided = any(pieces)
    while steps > 0:
        if slab.since == slab.halo:
            sl, sr = slab.halo_out()
            rl, rr = ex.exchange(sl, sr, slab._buf["recv_left"], slab._buf["recv_right"])
            slab.halo_in(rl, rr)
        k = 1 if divided else min(steps, slab.halo - slab.since)
        slab.advance(k)
        steps -= k
        if divided:
            every = ex.gather(slab.particles_out())
            if slab.piece is not None:
                slab.particles_in(_concat(every))


def run_local(slabs, steps: int) -> None:
    """`steps` steps of all slabs of one channel held by this process (rank
    order), exchanging in memory as run_dist does: the ranks of one channel
    emulated in lock step, with every copy ordered by the host."""
    W = len(slabs)
    divided = any(s.piece is not None for s in slabs)
    while steps > 0:
        if slabs[0].since == slabs[0].halo:
            outs = [s.halo_out() for s in slabs]          # each slab's own send buffers
            for r, s in enumerate(slabs):
                s.halo_in(outs[(r - 1) % W][1], outs[(r + 1) % W][0])
        k = 1 if divided else min(steps, slabs[0].halo - slabs[0].since)
        for s in slabs:
            s.advance(k)
        steps -= k
        if divided:
            owned = _concat([s.particles_out() for s in slabs])
            for s in slabs:
                if s.piece is not None:
                    s.particles_in(owned)
