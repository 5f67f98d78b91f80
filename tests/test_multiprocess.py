"""The N > 1 path of bench.py on CPU: independent replicas (no collective on
the data path) whose timing is the slowest rank's, exchanged with one MAX
all-reduce.  Two gloo ranks on 127.0.0.1 stand in for two GPUs."""
import os
import socket

import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        ms = [12.5, 20.0][rank]  # this rank's own timed region
        slowest = bench.max_over_ranks(ms)
        value = bench.whole_job_gbs(1_000_000_000, 10, ws, slowest)
        q.put((r, local, ws, slowest, value))
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, (rank, local, ws, slowest, value) in enumerate(got):
        assert rank == r and local == r and ws == 2
        assert slowest == 20.0  # every rank reports the slowest rank's time
        # 2 replicas x 10 steps x 1 GB in 20 ms
        assert value == pytest.approx(2 * 10 * 1.0 / 20e-3)


def test_single_process_needs_no_collective():
    assert not td.is_initialized()
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.whole_job_gbs(2_000_000_000, 5, 1, 10.0) == pytest.approx(1000.0)
