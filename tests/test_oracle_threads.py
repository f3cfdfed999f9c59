"""The oracle's all-cores timing build (OpenMP over LB nodes, particle
streaming and redraw; the CPU baseline and the reference arm of bench.py)
computes exactly what the single-threaded parity build computes: no loop it
shares out has a reduction or an order-dependent update.  Not GPU."""
import numpy as np
import pytest

import oracle as O
from tests import inputs

FIELDS = ("POPS", "RHO", "U", "PART_POS", "PART_VEL", "PART_HOME", "PART_CELL", "CELL_VCM", "WINDOW_MEAN")


@pytest.mark.parametrize("case", ["2d", "3d", "2d_resample", "2d_at"])
def test_threaded_build_equals_the_parity_build(case):
    if case == "3d":
        cfg = inputs.small_3d(precision=0)
    elif case == "2d_resample":
        cfg = inputs.small_2d(precision=0, resample_density=1)
    elif case == "2d_at":
        cfg = inputs.small_2d(precision=0, collision=1)
    else:
        cfg = inputs.small_2d(precision=0)
    sims = []
    for omp in (False, True):
        s = O.OracleSim(cfg["params"], omp=omp)
        s.set_region(*cfg["region"])
        s.step(12)
        sims.append(s)
    serial, threaded = sims
    for f in FIELDS:
        assert np.array_equal(serial.get(f), threaded.get(f)), f
    assert np.array_equal(serial.get("DIAG"), threaded.get("DIAG"))
