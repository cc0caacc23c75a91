"""The N > 1 path of bench.py on the CPU: two gloo ranks, each with its own
problem (same operator, fresh noise), gather their per-rank timings and the
whole-job throughput is the sum of all ranks' iterations over the slowest
rank's time (weak scaling, no data-path collective)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as wl
    p = bench.rank_problem(wl.make("ct64_sflsqr"), rank, wl, np)
    # a stand-in for the timed region: rank r "takes" 10 + r ms for 7 + r iterations
    per_rank = bench.gather_rank_values([10.0 + rank, 7 + rank], world, "cpu")
    t_max, total, value = bench.aggregate(per_rank, steps=3)
    bs = bench.gather_rank_values([float(np.linalg.norm(p.b)), float(p.noise_norm[0])], world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, per_rank, t_max, total, value, bs))


def test_two_gloo_ranks_aggregate_like_the_bench():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, per_rank, t_max, total, value, bs in res:
        assert per_rank == [[10.0, 7.0], [11.0, 8.0]]          # both ranks see every rank's values
        assert t_max == 11.0 and total == (7 + 8) * 3
        assert value == pytest.approx(45 / 0.011)
        assert bs[0] != bs[1]                                   # independent right-hand sides
        assert bs[0][1] == pytest.approx(bs[1][1], rel=0.05)    # same noise level
    assert res[0][1:] == res[1][1:]


def test_single_rank_aggregate():
    per_rank = bench.gather_rank_values([5.0, 10], 1, "cpu")
    assert bench.aggregate(per_rank, steps=2) == (5.0, 20, 4000.0)
