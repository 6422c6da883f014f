"""The N > 1 host path of bench.py on CPU: world size 2 over gloo (no GPU).

Each rank is an independent replica (pings do not shard further and need no data-path
collective); the only cross-rank steps are the barrier and the max-over-ranks timing,
and rank 0 alone reports. These run the same functions bench.py uses."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


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
        got_ws, got_rank, got_local = bench.dist_setup()
        # per-rank timings differ; every rank sees the slowest
        t = bench.max_over_ranks(10.0 + 5.0 * rank, got_ws)
        rate = bench.whole_job_rate(got_ws, 30, t)
        dist.barrier()
        out[rank] = (got_ws, got_rank, got_local, t, rate)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    assert out[0][:3] == (2, 0, 0) and out[1][:3] == (2, 1, 1)
    assert out[0][3] == out[1][3] == 15.0
    assert out[0][4] == out[1][4] == 2 * 30 / 15.0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse
    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    bench.run_reference(args, 2, 1)  # rank 1: returns at once, prints nothing
    assert capsys.readouterr().out == ""
