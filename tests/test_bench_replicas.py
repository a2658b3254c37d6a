"""Host logic of the bench's multi-process path (independent replicas, one per
GPU): rank parsing, the max over ranks of the timed region and the whole-job
aggregate, run as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    w, r, lr = bench.rank_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        elapsed = 1.0 + 0.5 * r  # rank 1 is the slow replica
        dist.barrier()
        t = bench.max_over_ranks(elapsed, dist, "cpu")
        v = bench.replica_value(1000, 10, w, t)
        dist.barrier()
        out[r] = (w, r, lr, t, v)
    finally:
        dist.destroy_process_group()


def test_rank_env_defaults_and_torchrun():
    assert bench.rank_env({}) == (1, 0, 0)
    assert bench.rank_env({"WORLD_SIZE": "4", "RANK": "3", "LOCAL_RANK": "1"}) == (4, 3, 1)


def test_single_process_value():
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.replica_value(100, 4, 1, 2.0) == 200.0


def test_two_gloo_replicas_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        for p in procs:
            if p.is_alive():
                p.kill()
                pytest.fail("a gloo rank did not finish")
            assert p.exitcode == 0
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (w, rr, lr, t, v) in res.items():
        assert (w, rr, lr) == (2, r, r)
        assert t == 1.5                           # max over the two ranks
        assert v == pytest.approx(1000 * 10 * 2 / 1.5)  # both replicas' cell-steps
