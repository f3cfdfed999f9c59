"""The paper's coupled LB-MPCD-AT channel (Sec. 3.2, Table 1 row 2) on the
GPU in binary32: a 30-row Poiseuille channel, LB nu = 0.167 (tau = 1), the
MPCD-AT region on the 30 central columns with 1000 particles per cell and kT
from Eq. 7 for the same viscosity, one-way coupled through 2-column buffers
(the paper's scheme).  The LB starts on its steady profile; after the MPCD
has relaxed, its time-averaged profile must reconnect with the LB one, i.e.
follow the analytic parabola.  The force is 5e-5 instead of Table 1's 5e-4
(Mach 0.6 on the LB side)."""
import numpy as np
import pytest

import oracle as O
from oracle import transport as T
from tests.test_gpu_parity import lb  # noqa: F401

pytestmark = pytest.mark.gpu


def test_coupled_mpcd_at_channel_table1_row2(lb):
    nx, H, ppc, nu, g = 90, 30, 1000, 1.0 / 6.0, 5e-5
    ny = H + 2
    kT = T.at_kT_for_viscosity(nu, ppc, 1.0)
    assert abs(kT - 0.17) < 0.01
    p = dict(lattice=9, nx=nx, ny=ny, nz=1, tau=0.5 + 3 * nu, force=(g, 0.0, 0.0), refine=1, ppc=ppc,
             alpha=0.0, kT=kT, mass=1.0, coupling_width=2, precision=1, feedback=0, window=100, seed=77,
             collision=1)
    sim = lb.Lbmpcd(p)
    sim.set_region(0, 30, 60)
    yc = np.arange(ny) + 0.5
    u = np.where((yc > 1) & (yc < ny - 1), g * (yc - 1) * (ny - 1 - yc) / (2 * nu), 0.0)
    f = np.stack([O.feq(9, 1.0, [ui, 0.0, 0.0]) for ui in u])
    sim.set("POPS", np.repeat(f.T[:, :, None], nx, axis=2).ravel())
    sim.step(12000)                       # > 2 H^2 / nu: the MPCD start-up has decayed
    mom, cnt = np.zeros(H), np.zeros(H)
    mom_c, cnt_c = np.zeros(H), np.zeros(H)
    for _ in range(300):
        sim.step(10)
        h = sim.get("PART_HOME").reshape(-1, 3)
        v = sim.get("PART_VEL").reshape(-1, 3)
        mom += np.bincount(h[:, 1], weights=v[:, 0], minlength=H)
        cnt += np.bincount(h[:, 1], minlength=H)
        mid = (h[:, 0] >= 10) & (h[:, 0] < 20)           # the 10 central columns, far from the buffers
        mom_c += np.bincount(h[mid, 1], weights=v[mid, 0], minlength=H)
        cnt_c += np.bincount(h[mid, 1], minlength=H)
    y = np.arange(H) + 0.5
    ua = g * y * (H - y) / (2 * nu)
    err = np.linalg.norm(mom / cnt - ua) / np.linalg.norm(ua)
    err_c = np.linalg.norm(mom_c / cnt_c - ua) / np.linalg.norm(ua)
    ul = sim.get("U").reshape(3, ny, nx)[0, 1:-1, :].mean(1)
    err_lb = np.linalg.norm(ul - ua) / np.linalg.norm(ua)
    print(f"coupled channel, N = {ppc}: rel. L2 against the parabola: MPCD region {err:.4f}, "
          f"central columns {err_c:.4f}, LB {err_lb:.2e}")
    assert err_lb < 1e-3
    assert err < 0.03 and err_c < 0.04
    sim.close()
