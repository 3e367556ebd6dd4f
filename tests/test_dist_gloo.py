"""The multi-process host logic on CPU: two gloo ranks on 127.0.0.1 check the
problem sharding of the batched path (every problem on exactly one rank) and the
whole-job reductions (units summed over ranks, time maximised over ranks) that
the benchmark uses for one-process-per-GPU runs."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    from paper_1009_3457_gb300 import dist as fdist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert fdist.world() == (world, rank)
        mine = fdist.shard(256, rank, world)
        # units: this rank's problems (their indices summed, so the sum is checkable); time: rank-dependent
        units = float(sum(mine))
        seconds = 1.0 + rank
        total = fdist.sum_over_ranks(units)
        slowest = fdist.max_over_ranks(seconds)
        rate = fdist.job_rate(units, seconds)
        out.put((rank, mine, total, slowest, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_shard_and_reductions_over_gloo_ranks(world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = sorted(i for _, mine, _, _, _ in res for i in mine)
    assert got == list(range(256))  # each problem on exactly one rank
    for rank, mine, total, slowest, rate in res:
        assert mine == list(range(rank, 256, world))
        assert total == float(sum(range(256)))
        assert slowest == float(world)  # 1 + (world - 1)
        assert rate == pytest.approx(sum(range(256)) / world)


def test_single_process_defaults():
    from paper_1009_3457_gb300 import dist as fdist

    assert fdist.world() == (1, 0)
    assert fdist.max_over_ranks(3.5) == 3.5 and fdist.sum_over_ranks(2.0) == 2.0
    assert fdist.job_rate(10.0, 2.0) == 5.0
    with pytest.raises(ValueError):
        fdist.shard(10, 2, 2)
