"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds workload descriptions and seeded random states only: no
step of the method's arithmetic lives here.  Each workload is a plane channel
(periodic in x and z, walls in y) with an MPCD sub-region of whole LB columns,
the structure of the paper's Poiseuille tests (Sec. 3) at the sizes of the
five benchmark workloads.
"""
from __future__ import annotations

import math

import numpy as np

DEG = math.pi / 180.0

# 2D Poiseuille channel, FP64: D2Q9 64x32, tau 1, g 1e-6; MPCD x in [24,40) at
# r = 1, 10 particles per cell, kT 1e-4, SRD 130 deg, 2-column coupling buffer.
CHANNEL_64x32_FP64 = dict(
    params=dict(lattice=9, nx=64, ny=32, nz=1, tau=1.0, force=(1e-6, 0.0, 0.0), refine=1,
                ppc=10, alpha=130 * DEG, kT=1e-4, mass=1.0, coupling_width=2, precision=0,
                feedback=1, window=100, resample_density=0, seed=1),
    region=(24, 40), steps=2000)

# 2D channel, FP32: D2Q9 2048x512, tau 0.8, g 1e-7; MPCD on the central 256
# LB columns at r = 2 (512 x 1020 cells, ~5.2M particles).
CHANNEL_2048x512_FP32 = dict(
    params=dict(lattice=9, nx=2048, ny=512, nz=1, tau=0.8, force=(1e-7, 0.0, 0.0), refine=2,
                ppc=10, alpha=130 * DEG, kT=1e-4, mass=1.0, coupling_width=2, precision=1,
                feedback=1, window=100, resample_density=0, seed=2),
    region=(896, 1152), steps=20000)

# 3D slab channel, FP32: D3Q19 256x128x128, tau 0.9, g 5e-8; MPCD slab
# x in [112,144) at r = 2 (64 x 252 x 256 cells, ~41M particles), SRD 120 deg.
SLAB_256x128x128_FP32 = dict(
    params=dict(lattice=19, nx=256, ny=128, nz=128, tau=0.9, force=(5e-8, 0.0, 0.0), refine=2,
                ppc=10, alpha=120 * DEG, kT=1e-4, mass=1.0, coupling_width=2, precision=1,
                feedback=1, window=100, resample_density=0, seed=3),
    region=(112, 144), steps=5000)


def with_(cfg: dict, **over) -> dict:
    """Copy of a workload with parameter overrides (region/steps kept)."""
    out = dict(cfg)
    out["params"] = dict(cfg["params"], **over)
    return out


def small_2d(**over) -> dict:
    """A few-tile 2D case with a ragged tail: 70 x 22 nodes, MPCD x in [20,43) at r = 2."""
    p = dict(lattice=9, nx=70, ny=22, nz=1, tau=0.85, force=(2e-5, 0.0, 0.0), refine=2,
             ppc=7, alpha=130 * DEG, kT=1e-4, mass=1.0, coupling_width=2, precision=0,
             feedback=1, window=5, resample_density=0, seed=11)
    p.update(over)
    return dict(params=p, region=(20, 43), steps=5)


def small_3d(**over) -> dict:
    """A small 3D slab: D3Q19 21 x 12 x 10 nodes, MPCD x in [6,15) at r = 2."""
    p = dict(lattice=19, nx=21, ny=12, nz=10, tau=0.9, force=(1e-5, 0.0, 2e-6), refine=2,
             ppc=5, alpha=120 * DEG, kT=1e-4, mass=1.0, coupling_width=2, precision=0,
             feedback=1, window=4, resample_density=0, seed=13)
    p.update(over)
    return dict(params=p, region=(6, 15), steps=3)


def ensemble_replicas(n: int = 64, seed: int = 4) -> list:
    """Uneven replica set: Ny in {16,32,64,128}, Nx = 4 Ny, r in {1,2,4},
    tau ~ U[0.6,1.2], g ~ U[1e-7,1e-6], 5..20 particles per cell, distinct
    seeds; MPCD on the central Nx/4 columns."""
    rng = np.random.default_rng(seed)
    reps = []
    for k in range(n):
        ny = int(rng.choice([16, 32, 64, 128]))
        nx = 4 * ny
        p = dict(lattice=9, nx=nx, ny=ny, nz=1, tau=float(rng.uniform(0.6, 1.2)),
                 force=(float(rng.uniform(1e-7, 1e-6)), 0.0, 0.0), refine=int(rng.choice([1, 2, 4])),
                 ppc=int(rng.integers(5, 21)), alpha=130 * DEG, kT=1e-4, mass=1.0,
                 coupling_width=2, precision=1, feedback=1, window=100, resample_density=0,
                 seed=1000 + k)
        reps.append(dict(params=p, region=(nx // 2 - nx // 8, nx // 2 + nx // 8)))
    return reps


def perturbed_populations(q: int, shape, weights, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Populations w_i (1 + amp * U(-1,1)), layout [q][nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    base = np.asarray(weights, dtype=np.float64).reshape(q, 1, 1, 1)
    return base * (1.0 + amp * rng.uniform(-1.0, 1.0, size=(q,) + tuple(shape)))


def random_velocities(n: int, dim: int, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = np.zeros((n, 3))
    v[:, :dim] = rng.normal(0.0, sigma, size=(n, dim))
    return v


def grid_offsets(n: int, dim: int, seed: int) -> np.ndarray:
    """Offsets in [0,1) on the 2^-24 grid (exact in binary32 and binary64)."""
    rng = np.random.default_rng(seed)
    o = np.zeros((n, 3))
    o[:, :dim] = rng.integers(0, 1 << 24, size=(n, dim)) / float(1 << 24)
    return o
