"""The N > 1 path of bench.py on the CPU: two gloo ranks, each an independent
replica with its own step time. Every rank must see the slowest rank's time
(max over ranks), and the whole-job rate is the units of all ranks over that
time."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    local_seconds = [2.0, 3.5][rank]
    slowest = bench.max_over_ranks(local_seconds, dist, "cpu")
    rate = bench.job_throughput(8, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.spawn(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        res = json.load(open(tmp_path / f"rank{rank}.json"))
        assert res["slowest"] == 3.5
        assert abs(res["rate"] - 8 * 2 / 3.5) < 1e-12


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.job_throughput(4, 1, 2.0) == 2.0
