"""The multi-rank bookkeeping of bench.py on CPU (world size 2, gloo): every
rank gets the slowest rank's time, the whole-job rate counts all ranks'
steps over that time, and the ranks run distinct replicas.  Not GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + 0.5 * rank, world, "cpu")
        out[rank] = (t, bench.job_rate(100, world, t), bench.rank_params({"seed": 2, "nx": 8}, rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        t, rate, params = res[r]
        assert t == 1.5
        assert rate == pytest.approx(2 * 100 / 1.5)
        assert params == {"seed": 2 + 1000 * r, "nx": 8}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.25, 1, "cpu") == 0.25
    assert bench.job_rate(64, 1, 0.5) == 128.0
