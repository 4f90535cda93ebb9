"""Host logic of the replicated multi-GPU run, on CPU with two gloo ranks.

One system does not shard (the block projections are sequential on one x), so
``bench.py --gpus N`` runs N replicas: each rank solves its own system and the
step time is the maximum over ranks.  This test runs that host logic (rank ->
system seed, max over ranks, barrier) as two processes with the gloo backend;
no GPU and no solver call is involved.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    seed = bench.replica_seed(r)
    # a per-rank step time that differs between ranks
    t = 10.0 + 3.5 * r
    t_max = bench.max_over_ranks(t, dist, "cpu")
    seeds = [None] * w
    dist.all_gather_object(seeds, seed)
    dist.barrier()
    out.put((r, w, local, seed, t_max, seeds))
    dist.destroy_process_group()


def test_two_replicas_have_distinct_systems_and_max_step_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == world and r[2] == r[0] for r in res)
    # independent systems: distinct seeds on every rank
    assert len(set(res[0][5])) == world
    # every rank reports the job's step time: the slowest rank's
    assert all(r[4] == 10.0 + 3.5 * (world - 1) for r in res)


def test_single_process_max_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.max_over_ranks(4.25, None, "cpu") == 4.25
    assert bench.replica_seed(0) == 1
