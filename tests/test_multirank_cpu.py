"""The N > 1 host path of bench.py on CPU: two gloo ranks, one per process.

With several GPUs bench.py runs independent replicas (one tensor per rank);
the process group carries only the barrier and the max of the per-rank
times, and the reported value is the bytes of all ranks over that max.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    w, r, local = bench.dist_setup(world)
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(w, 1.5 + rank)  # per-rank seconds; the job takes the slowest
    nbytes = 1e9
    value = w * nbytes / t / 1e9               # whole-job GB/s, as bench.py reports it
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{t} {value}")
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    for rank in range(world):
        t, value = map(float, (tmp_path / f"rank{rank}.txt").read_text().split())
        assert t == 2.5
        assert value == pytest.approx(world / 2.5)
