"""The replicas path of bench.py (one simulation per rank, no data-path
collective) on two gloo ranks on the CPU: the per-rank seeds differ, the
job time is the slowest rank's, the whole-job value counts every rank's
particles, and batched simulations are split without overlap."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = 1.5 + rank                       # the slower rank decides
    t = bench.max_over_ranks(seconds, world)
    out.put((rank, bench.rank_seed(100, rank), t,
             bench.job_value(world, 512 ** 3, 40, t),
             bench.shard(list(range(64)), rank, world)))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    seeds = {r[1] for r in res}
    assert seeds == {100, 101}
    assert all(r[2] == pytest.approx(2.5) for r in res)
    assert all(r[3] == pytest.approx(2 * 512 ** 3 * 40 / 2.5) for r in res)
    shards = [set(r[4]) for r in res]
    assert not (shards[0] & shards[1]) and (shards[0] | shards[1]) == set(range(64))

