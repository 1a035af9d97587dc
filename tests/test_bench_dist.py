"""The multi-rank host logic of bench.py on CPU with gloo, world size 2 (replicas only: no data-path
collective; the ranks meet only for the barrier and the max over ranks of the timed interval)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        bench.barrier(world)
        mx = bench.barrier_max(world, 10.0 + 5.0 * rank)  # rank 1 is the slow one
        val = bench.job_value(world, 1000.0, 4, mx)
        os.environ["RANK"] = str(rank)
        ref = bench.run_reference(type("A", (), {"workload": "elastic_vibration", "warmup": 3, "steps": 1, "preroll": 2})(), rank,
                                  world) if rank == 1 else "skipped"
        out.put((rank, mx, val, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_report_the_whole_job():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val, ref in res:
        assert mx == 15.0  # the slowest rank's time on every rank
        assert val == pytest.approx(2 * 1000.0 * 4 / 15e-3)
    assert res[1][3] is None  # only rank 0 runs and prints the reference arm
