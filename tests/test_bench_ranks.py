"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2) check the max-over-ranks
timing, the summed work units and the sharding of independent instances (every instance exactly
once), as a torchrun launch of `bench.py --gpus 2` uses them."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    try:
        # rank r took 10 + r ms for 1000 (r + 1) units: the job's time is the slowest rank's
        (ms,), (units,) = bench.reduce_over_ranks(dist, [10.0 + rank], [1000.0 * (rank + 1)], "cpu")
        mine = bench.shard(list(range(48)), rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out.put((rank, ms, units, sorted(sum(gathered, []))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, everything in res:
        assert ms == 11.0                      # max over ranks
        assert units == 3000.0                 # sum over ranks
        assert everything == list(range(48))   # every instance on exactly one rank


def test_single_process_reduction_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, [3.5, 1.0], [7, 2], "cpu") == ([3.5, 1.0], [7.0, 2.0])
    assert bench.shard(list(range(5)), 0, 1) == list(range(5))
