"""The N > 1 path of the benchmark on CPU: two gloo ranks, each timing its own replica, agree on the
slowest rank's time and on the whole job's rate; every rank draws a different system."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1406_5802_gb300 import ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 37.5 * rank  # rank 1 is the slower replica
        slowest = ranks.max_over_ranks(local_ms, world)
        rate = ranks.whole_job_rate(5, world, slowest / 1e3)
        out[rank] = (slowest, rate, ranks.system_seed(1000, rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in (0, 1):
        slowest, rate, _ = res[rank]
        assert slowest == 137.5  # the maximum, seen by both ranks
        assert rate == pytest.approx(5 * world / 0.1375)  # all ranks' solves over the slowest time
    assert res[0][2] == 1000 and res[1][2] == 1000 + ranks.SEED_STRIDE  # one system per rank


def test_single_rank_needs_no_process_group():
    assert ranks.max_over_ranks(12.5, 1) == 12.5
    assert ranks.whole_job_rate(10, 1, 2.0) == 5.0
    with pytest.raises(ValueError):
        ranks.whole_job_rate(10, 1, 0.0)
    with pytest.raises(ValueError):
        ranks.system_seed(1, -1)
