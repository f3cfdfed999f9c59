"""Training data, training and evaluation of the learned MPCD->LB closure on
the GPU.

The data come from the coupled method itself: channels run with
``feedback = 2`` and no parameters loaded (one-way coupling plus sampling);
every ``every`` steps the network input of each replica (the last 8 strip
frames, ``CLOSURE_IN``) and its target (the 500-step moving average,
``CLOSURE_TARGET``) are copied into device tensors.  Each channel starts
from the steady Poiseuille profile of its LB viscosity (populations from
``U``, particle velocities shifted by the profile), so that the samples are
taken near the statistically steady state the closure serves.

Training runs the library's tcgen05 forward/backward kernels and its Adam
step (``Net.train_step``); evaluation compares the trained network and the
plain 8-frame mean against the same target.  Torch is used for device memory
and random batch indices only.
"""
from __future__ import annotations

import math

import numpy as np

from . import Lbmpcd, Net, load_library

DEG = math.pi / 180.0


def channel(ny: int, g: float, seed: int, nx: int = 128, region_cols: int = 64, tau: float = 0.8,
            refine: int = 2, ppc: int = 10, kT: float = 1e-4, precision: int = 1) -> dict:
    """A 2D channel of the training family (the 2048 x 512 channel's
    parameters at another size): D2Q9, walls in y, MPCD on the central
    ``region_cols`` LB columns at refinement 2, learned-closure sampling on."""
    x0 = (nx - region_cols) // 2
    p = dict(lattice=9, nx=nx, ny=ny, nz=1, tau=tau, force=(g, 0.0, 0.0), refine=refine, ppc=ppc,
             alpha=130 * DEG, kT=kT, mass=1.0, coupling_width=2, precision=precision, feedback=2,
             window=100, resample_density=0, seed=seed)
    return dict(params=p, region=(x0, x0 + region_cols))


def poiseuille(y, ny: int, tau: float, g: float):
    """Steady profile between the half-way walls y = 1 and y = ny - 1."""
    nu = (tau - 0.5) / 3.0
    return g / (2.0 * nu) * (y - 1.0) * (ny - 1.0 - y)


def matched_tau(ppc: float, kT: float, alpha: float, refine: int, mass: float = 1.0) -> float:
    """LB relaxation time whose kinematic viscosity (tau - 1/2) / 3 equals that
    of the 2D SRD fluid of the coupled region (kinetic-theory form: kinetic
    part kT dt / m (M / (s (1 - cos 2 alpha)) - 1/2), collisional part
    a^2 (1 - cos alpha) s / (12 M dt), s = M - 1 + e^-M, cell size a =
    1 / refine, dt = 1).  With it the coupled channel's steady state is the
    analytic Poiseuille profile of that viscosity."""
    M = float(ppc)
    s = M - 1.0 + math.exp(-M)
    a = 1.0 / refine
    kin = kT / mass * (M / (s * (1.0 - math.cos(2.0 * alpha))) - 0.5)
    col = a * a * (1.0 - math.cos(alpha)) * s / (12.0 * M)
    return 0.5 + 3.0 * (kin + col)


def training_channels(n: int, seed: int, ny_choices=(64, 128, 256, 512), g_range=(1e-7, 1e-6),
                      umax: float = 0.05, **kw) -> list:
    """n channels: Ny drawn from ny_choices, g log-uniform in g_range and
    lowered where the centreline velocity would exceed umax (low Mach)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        ny = int(ny_choices[k % len(ny_choices)])
        g = float(np.exp(rng.uniform(np.log(g_range[0]), np.log(g_range[1]))))
        tau = kw.get("tau", 0.8)
        cap = umax / poiseuille(ny / 2.0, ny, tau, 1.0)
        out.append(channel(ny, min(g, cap), seed=10_000 * seed + k, **kw))
    return out


def start_from_poiseuille(sim: Lbmpcd, replica: int, cfg: dict) -> None:
    p = cfg["params"]
    nx, ny, r = p["nx"], p["ny"], p["refine"]
    g, tau = p["force"][0], p["tau"]
    U = np.zeros((3, 1, ny, nx))
    yc = np.arange(ny) + 0.5
    prof = np.where((yc > 1) & (yc < ny - 1), poiseuille(yc, ny, tau, g), 0.0)
    U[0, 0] = prof[:, None]
    sim.set("U", U, replica)
    vel = sim.get("PART_VEL", replica).reshape(-1, 3)
    home = sim.get("PART_HOME", replica).reshape(-1, 3)
    pos = sim.get("PART_POS", replica).reshape(-1, 3)
    y = 1.0 + (home[:, 1] + pos[:, 1]) / r
    vel[:, 0] += poiseuille(y, ny, tau, g)
    sim.set("PART_VEL", vel, replica)


def generate(channels: list, spinup: int, samples: int, every: int):
    """Run the channels in one handle and collect (X, T): X (N, 16, 16, 24) and
    T (N, 16, 16, 3) float32 CUDA tensors, N = samples x patches of all
    channels."""
    import torch
    sim = Lbmpcd([c["params"] for c in channels])
    for r, c in enumerate(channels):
        sim.set_region(r, *c["region"])
    for r, c in enumerate(channels):
        start_from_poiseuille(sim, r, c)
    sizes = [sim_size(sim, r) for r in range(len(channels))]
    P = sum(sizes)
    X = torch.empty(samples * P, 16, 16, 24, dtype=torch.float32, device="cuda")
    T = torch.empty(samples * P, 16, 16, 3, dtype=torch.float32, device="cuda")
    buf_x = torch.empty(max(sizes) * 256 * 24, dtype=torch.float64, device="cuda")
    buf_t = torch.empty(max(sizes) * 256 * 3, dtype=torch.float64, device="cuda")
    sim.step(spinup)
    o = 0
    for s in range(samples):
        sim.step(every)
        for r, pr in enumerate(sizes):
            bx, bt = buf_x[: pr * 256 * 24], buf_t[: pr * 256 * 3]
            sim.get("CLOSURE_IN", r, out=bx)
            sim.get("CLOSURE_TARGET", r, out=bt)
            X[o:o + pr] = bx.view(pr, 16, 16, 24).float()
            T[o:o + pr] = bt.view(pr, 16, 16, 3).float()
            o += pr
    torch.cuda.synchronize()
    sim.close()
    return X, T


def sim_size(sim: Lbmpcd, replica: int) -> int:
    """Closure patches of one replica."""
    from . import lbmpcd_field_size
    return lbmpcd_field_size(sim._h, replica, "CLOSURE_TARGET") // 768


def train(X, T, steps: int, batch: int = 32, lr: float = 1e-3, seed: int = 0, theta=None, log_every: int = 0):
    """Adam on random batches of (X, T) with a cosine-decayed rate; returns
    (parameters as float32 numpy, per-step losses)."""
    import torch
    net = Net(batch)
    n = int(load_library().lbmpcd_net_num_params())
    if theta is None:
        theta = init_params(seed)
    net.set_params(theta)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    losses = []
    N = X.shape[0]
    for k in range(steps):
        idx = torch.randint(0, N, (batch,), device="cuda", generator=gen)
        xb, tb = X[idx].contiguous(), T[idx].contiguous()
        rate = lr * 0.5 * (1.0 + math.cos(math.pi * k / max(steps, 1)))
        losses.append(net.train_step(xb, tb, max(rate, 1e-3 * lr)))
        if log_every and (k % log_every == 0 or k == steps - 1):
            print(f"step {k}: loss {losses[-1]:.5f}")
    theta = net.get_params()
    net.close()
    assert theta.size == n
    return theta, np.asarray(losses)


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, the last layer scaled by 0.1 (the
    network starts close to the plain 8-frame mean it corrects; the
    correction is centred along y in each patch column, so the column means
    stay those of the 8-frame mean)."""
    rng = np.random.default_rng(seed)
    parts = []
    layers = [(24, 64), (64, 64), (64, 64), (64, 3)]
    for li, (ci, co) in enumerate(layers):
        std = math.sqrt(2.0 / (9 * ci)) * (0.1 if li == len(layers) - 1 else 1.0)
        parts.append(rng.normal(0.0, std, size=co * 9 * ci))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def evaluate(theta, X, T, chunk: int = 256) -> dict:
    """RMS error per field (density deviation, u_x, u_y in thermal units) of
    the network and of the plain 8-frame mean against the target, and their
    ratio (the gain)."""
    import torch
    net = Net(chunk)
    net.set_params(theta)
    se_net = torch.zeros(3, dtype=torch.float64, device="cuda")
    se_m8 = torch.zeros(3, dtype=torch.float64, device="cuda")
    y = torch.empty(chunk, 16, 16, 3, dtype=torch.float32, device="cuda")
    N = X.shape[0]
    for o in range(0, N, chunk):
        xb = X[o:o + chunk].contiguous()
        tb = T[o:o + chunk]
        P = xb.shape[0]
        net.forward(xb, y[:P])
        m8 = xb.view(P, 16, 16, 8, 3).mean(dim=3)
        se_net += ((y[:P] - tb).double() ** 2).sum(dim=(0, 1, 2))
        se_m8 += ((m8 - tb).double() ** 2).sum(dim=(0, 1, 2))
    net.close()
    cnt = N * 256
    rn = (se_net / cnt).sqrt().cpu().numpy()
    rm = (se_m8 / cnt).sqrt().cpu().numpy()
    return dict(rmse_net=rn, rmse_mean8=rm, gain=rm / rn)
