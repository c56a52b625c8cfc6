"""The multi-rank bench path on CPU (gloo, world size 2): every rank renders its
own snapshot (distinct seeds), the slowest rank's time is the job's time and
the whole-job rate counts the units of all ranks.  No GPU is involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench.dist_env()
        t = bench.max_over_ranks(times[r], w, "cpu")
        out[r] = (t, bench.whole_job_rate(1000.0, w, t / 1e3), bench.replica_seed(r))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_units():
    ws, port = 2, _free_port()
    times = [12.5, 20.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, times, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    assert res[0][1] == pytest.approx(1000.0 * 2 / 0.020)
    assert res[0][2] != res[1][2]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
