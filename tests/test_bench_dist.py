"""Multi-process (world size 2, gloo on the CPU) checks of bench.py's replica timing: the job
time is the maximum over ranks and the metric divides it by the solves of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        mx = bench.max_over_ranks(1.5 + rank, ws, device="cpu")
        out[rank] = (env, mx)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_world_size_2():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    assert out[0][1] == out[1][1] == 2.5
    assert out[0][0] == (2, 0, 0) and out[1][0] == (2, 1, 1)


def test_seconds_per_solve_counts_every_rank():
    import bench
    # two ranks, 3 solves each, slowest rank 600 ms: 6 solves in 0.6 s
    assert bench.seconds_per_solve(600.0, 3, 2) == pytest.approx(0.1)
    assert bench.max_over_ranks(4.0, 1) == 4.0
