"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): each rank
runs its own replica; the job time is the slowest rank's and the whole-job
value counts every rank's cells.  No GPU is used."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, w = bench.dist_env()
        # rank r took 100 + 50 r ms for its steps
        total = bench.max_over_ranks(100.0 + 50.0 * r, w, device="cpu")
        value = bench.weak_value(w, cells=262_144, deposits=100, steps=10, total_ms=total)
        dist.barrier()
        q.put((r, w, total, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_all_cells():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for r, (rr, w, total, value) in enumerate(out):
        assert rr == r and w == world
        assert total == 150.0                           # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 262_144 * 100 * 10 / 0.150)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.weak_value(1, 10, 2, 3, 1000.0) == pytest.approx(60.0)
