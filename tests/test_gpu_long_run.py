"""Long runs on the GPU (GPU).

* The 64 x 32 FP64 channel (MPCD x in [24,40), r = 1, 10 particles per cell,
  two-way coupling) for its full 2000 steps, SRD and MPCD-AT: the MPCD
  velocity profile (x-averaged per fine row) and the LB profile, both
  time-averaged over the last 500 steps, match the oracle's within 1% L2.
  Binary64 with the oracle's own random numbers keeps the two runs on the
  same trajectory (binning is exact and the collision is linear in the
  velocities), so the profiles agree far below 1%; at this channel's kT and g
  a comparison of independent runs would need ~10^4 replicas to get below 1%
  (seed-to-seed scatter of one run: ~86% for the LB profile, measured with the
  oracle).
* Binary32 production precision, standalone MPCD Poiseuille flows: the fitted
  viscosity matches Eq. 7 (MPCD-AT) and the kinetic-theory SRD form, the same
  pins the oracle is held to."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import transport as T
from tests import inputs
from tests.test_gpu_parity import lb  # noqa: F401

pytestmark = pytest.mark.gpu


def _profiles(sim, get, p, region, Hy):
    h = get(sim, "PART_HOME").reshape(-1, 3)
    v = get(sim, "PART_VEL").reshape(-1, 3)
    mom = np.bincount(h[:, 1], weights=v[:, 0], minlength=Hy)
    cnt = np.bincount(h[:, 1], minlength=Hy)
    u = get(sim, "U").reshape(3, p["ny"], p["nx"])[0, 1:-1, :].mean(1)
    return mom, cnt, u


@pytest.mark.parametrize("collision", [0, 1])
def test_long_run_fp64_tracks_oracle(lb, collision):
    cfg = inputs.with_(inputs.CHANNEL_64x32_FP64, collision=collision)
    p, region, steps = cfg["params"], cfg["region"], cfg["steps"]
    Hy = (p["ny"] - 2) * p["refine"]
    g = lb.Lbmpcd(p)
    g.set_region(0, *region)
    o = O.OracleSim(p)
    o.set_region(*region)
    acc = {}
    for name, sim, get in (("gpu", g, lambda s, f: s.get(f)), ("oracle", o, lambda s, f: s.get(f))):
        sim.step(steps - 500)
        mom, cnt, ul = np.zeros(Hy), np.zeros(Hy), np.zeros(p["ny"] - 2)
        for _ in range(100):
            sim.step(5)
            a, b, c = _profiles(sim, get, p, region, Hy)
            mom += a
            cnt += b
            ul += c
        acc[name] = (mom / cnt, ul / 100)
    e_mpcd = np.linalg.norm(acc["gpu"][0] - acc["oracle"][0]) / np.linalg.norm(acc["oracle"][0])
    e_lb = np.linalg.norm(acc["gpu"][1] - acc["oracle"][1]) / np.linalg.norm(acc["oracle"][1])
    vmax = float(np.max(np.abs(g.get("PART_VEL") - o.get("PART_VEL"))))
    print(f"collision {collision}: {steps} steps, rel. L2 MPCD profile {e_mpcd:.2e}, LB profile {e_lb:.2e}, "
          f"max |dv| at the end {vmax:.2e}")
    assert e_mpcd < 0.01 and e_lb < 0.01
    g.close()


@pytest.mark.parametrize("collision,kT,tol", [(1, 0.25, 0.03), (1, 0.05, 0.04), (0, 1.0, 0.06)])
def test_fp32_standalone_viscosity(lb, collision, kT, tol):
    """Channel H = 10 between half-way walls, 240 columns, periodic in x, no
    coupling buffer; 10 particles per cell, r = 1; g set for u_max = 0.15;
    10,000 steps after 1,000, profile every 10 steps."""
    alpha = math.radians(130.0)
    ppc, H, W = 10, 10, 240
    kin, col = T.at_viscosity(ppc, kT) if collision else T.srd_viscosity_2d(ppc, kT, alpha)
    nu = kin + col
    gacc = 8.0 * nu * 0.15 / H ** 2
    p = dict(lattice=9, nx=W, ny=H + 2, nz=1, tau=0.5 + 3.0 * nu, force=(gacc, 0.0, 0.0), refine=1, ppc=ppc,
             alpha=alpha, kT=kT, mass=1.0, coupling_width=0, precision=1, feedback=0, window=1,
             resample_density=0, seed=21, collision=collision)
    sim = lb.Lbmpcd(p)
    sim.set_region(0, 0, W)
    sim.step(1000)
    mom, cnt = np.zeros(H), np.zeros(H)
    for _ in range(1000):
        sim.step(10)
        h = sim.get("PART_HOME").reshape(-1, 3)
        v = sim.get("PART_VEL").reshape(-1, 3)
        mom += np.bincount(h[:, 1], weights=v[:, 0], minlength=H)
        cnt += np.bincount(h[:, 1], minlength=H)
    u = mom / cnt
    y = 1.0 + np.arange(H) + 0.5
    shape = (y - 1.0) * (H + 1.0 - y) / 2.0
    fit = gacc * np.sum(shape * shape) / np.sum(shape * u)
    print(f"collision {collision} kT {kT}: closed form {nu:.4f}, FP32 GPU fit {fit:.4f} ({fit / nu - 1:+.2%})")
    assert abs(fit / nu - 1.0) < tol
    sim.close()
