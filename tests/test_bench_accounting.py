"""The accounting of bench.py on CPU: the algorithmic bytes of a step (72 B
per fluid LB node, 40 B per particle, 24 B per collision cell), the kernel
launches it claims for a call, and the ncu traffic it takes from the
committed summary only while the kernel sources match the recorded hashes.
Not GPU."""
import hashlib
import os

import bench


def test_algorithmic_bytes_of_the_2048x512_channel():
    b = bench.algorithmic_bytes(bench.WORKLOAD["params"], bench.WORKLOAD["region"])
    # 2048 x 510 fluid nodes; 256 region columns at refinement 2 over 510 rows,
    # 10 particles per cell; collision cells one row more than home cells
    assert b["fluid_nodes"] == 2048 * 510
    assert b["particles"] == 512 * 1020 * 10 == 5_222_400
    assert b["cells"] == 512 * 1021
    step = 72 * b["fluid_nodes"] + 40 * b["particles"] + 24 * b["cells"]
    assert step == 296_644_608
    assert b["lb_rows"] + b["particle_pass"] + b["cell_items"] == step
    assert b["lb_pull"] == b["lb_rows"] + b["cell_items"]


def test_launch_count_of_a_20_step_call():
    # overlapped form, one chunk of 20 steps after 5 warm-up steps: one prep,
    # the chunk's first LB launch, three launches per step but the last, which
    # has two (particle pass, table)
    n, n_end, last_sort = bench.step_launches(5, 0, 20, 0, overlapped=True)
    assert n == 1 + 1 + 19 * 3 + 2 == 61
    assert n_end == 25 and last_sort == 0
    # serial form: two kernels per step
    n, _, _ = bench.step_launches(5, 0, 20, 0, overlapped=False)
    assert n == 1 + 20 * 2


def test_ncu_traffic_follows_the_source_hashes(tmp_path, monkeypatch):
    txt = open(bench.PROFILE_NOTE).read()
    vals = {}
    for ln in txt.splitlines():
        if ln.strip().startswith("- ") and ": " in ln:
            k, v = ln.strip()[2:].split(": ", 1)
            vals[k] = v
    pass_b = float(vals["dram_bytes_per_launch"])
    rows_b = float(vals["rows_dram_bytes_per_launch"])
    src = os.path.join(bench.ROOT, "paper_2004_00304_gb300", "csrc")
    current = all(vals.get(f + " sha256[:16]") == hashlib.sha256(open(os.path.join(src, f), "rb").read()).hexdigest()[:16]
                  for f in ("mpcd.cu", "lb.cu", "lb_core.cuh", "cell_core.cuh", "common.cuh", "kernels.h"))
    if current:
        assert bench.ncu_traffic_per_launch() == pass_b
        assert bench.ncu_traffic_per_launch(pair=True) == pass_b + rows_b
    # a summary whose recorded hash no longer matches gives no traffic
    stale = txt.replace(vals["lb.cu sha256[:16]"], "0" * 16)
    note = tmp_path / "note.md"
    note.write_text(stale)
    monkeypatch.setattr(bench, "PROFILE_NOTE", str(note))
    assert bench.ncu_traffic_per_launch() is None
    assert bench.ncu_traffic_per_launch(pair=True) is None
