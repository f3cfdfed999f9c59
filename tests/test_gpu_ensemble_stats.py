"""Long-run statistics of the binary32 path against the FP64 oracle (GPU).

The particle trajectories of the two implementations separate after a few
hundred steps (binary32 rounding of chaotic MPCD dynamics), so a long run is
compared through ensemble means, as the velocity profiles of the paper's
Sec. 3.1 are time averages: 64 replicas of the 64 x 32 channel (D2Q9,
tau = 1, MPCD on columns [24, 40) at r = 1 with ppc = 10, kT = 1e-4, SRD at
130 degrees, two-way coupling with W = 100) with distinct seeds run in one
binary32 handle and, independently, in the FP64 oracle; each side's profiles
are averaged over 100 samples 20 steps apart after 1000 steps, and over the
replicas:
  MPCD  mean particle velocity u_x per MPCD row,
  LB    velocity u_x per row averaged over all columns.
The two ensemble means must agree within 1 % relative L2.

Sizing by Eq. 8: one sample of an MPCD row mean has sigma = sqrt(kT / N) with
N = 16 columns x 10 particles = 160, i.e. 7.9e-4; with g = 5e-5 the profile
reaches ~0.02 at the centre by step 1000, so the 6400 correlated samples per
side (effective count reported below) bring the standard error of the
difference well under 1 %; the test also checks that it does, so that the
1 % bound resolves a real disagreement."""
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NREP, SPIN, NSAMP, EVERY = 64, 1000, 100, 20
REGION = (24, 40)


def channel(seed: int) -> dict:
    return dict(lattice=9, nx=64, ny=32, nz=1, tau=1.0, force=(5e-5, 0.0, 0.0), refine=1, ppc=10,
                alpha=np.radians(130.0), kT=1e-4, mass=1.0, coupling_width=2, precision=1, feedback=1,
                window=100, resample_density=0, seed=seed)


def profiles(home, vel, u, hy):
    """MPCD row means of u_x and the column-averaged LB u_x per fluid row."""
    y = home[:, 1]
    cnt = np.bincount(y, minlength=hy)
    mp_row = np.bincount(y, weights=vel[:, 0], minlength=hy) / np.maximum(cnt, 1)
    ny, nx = u.shape[1], u.shape[2]
    return mp_row, u[0, 1:ny - 1, :].mean(axis=1)


def oracle_replica(seed: int):
    """Sum and sum of squares (over the samples) of both profiles of one
    oracle replica, in FP64."""
    import oracle as O
    p = dict(channel(seed), precision=0)
    s = O.OracleSim(p)
    s.set_region(*REGION)
    s.step(SPIN)
    hy = p["ny"] - 2
    acc = np.zeros((2, 2, hy))
    for _ in range(NSAMP):
        s.step(EVERY)
        a, b = profiles(s.get("PART_HOME").reshape(-1, 3), s.get("PART_VEL").reshape(-1, 3),
                        s.get("U").reshape(3, p["ny"], p["nx"]), hy)
        acc[0, 0] += a; acc[1, 0] += a * a
        acc[0, 1] += b; acc[1, 1] += b * b
    return acc


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2004_00304_gb300 as mod
    return mod


def test_fp32_ensemble_mean_profiles_match_oracle(lb):
    seeds = [101 + 7 * k for k in range(NREP)]
    # the oracle replicas on the host cores (spawned workers: the parent holds a CUDA context)
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(processes=max(1, min(16, mp.cpu_count())))
    pending = pool.map_async(oracle_replica, seeds)

    p0 = channel(seeds[0])
    hy, ny, nx = p0["ny"] - 2, p0["ny"], p0["nx"]
    sim = lb.Lbmpcd([channel(s) for s in seeds])
    for k in range(NREP):
        sim.set_region(k, *REGION)
    sim.step(SPIN)
    gacc = np.zeros((NREP, 2, 2, hy))
    for _ in range(NSAMP):
        sim.step(EVERY)
        for k in range(NREP):
            a, b = profiles(sim.get("PART_HOME", k).reshape(-1, 3), sim.get("PART_VEL", k).reshape(-1, 3),
                            sim.get("U", k).reshape(3, ny, nx), hy)
            gacc[k, 0, 0] += a; gacc[k, 1, 0] += a * a
            gacc[k, 0, 1] += b; gacc[k, 1, 1] += b * b
    sim.close()
    oacc = np.array(pending.get(timeout=1800))
    pool.close()
    pool.join()

    for j, name in enumerate(("MPCD", "LB")):
        g_rep = gacc[:, 0, j] / NSAMP          # per-replica time means
        o_rep = oacc[:, 0, j] / NSAMP
        g_mean, o_mean = g_rep.mean(0), o_rep.mean(0)
        # standard error of each ensemble mean from the replica scatter
        se = np.sqrt(g_rep.var(0, ddof=1) / NREP + o_rep.var(0, ddof=1) / NREP)
        err = float(np.linalg.norm(g_mean - o_mean) / np.linalg.norm(o_mean))
        noise = float(np.linalg.norm(se) / np.linalg.norm(o_mean))
        print(f"{name}: rel L2 (binary32 GPU vs FP64 oracle ensemble means) {err:.4f}, "
              f"standard error of the difference {noise:.4f}")
        assert noise < 0.004, (name, noise)   # the comparison resolves 1 %
        assert err < 0.01, (name, err)
