"""Multi-rank host logic of the replica runs on CPU: world_size 2 over gloo.

Each rank reports different work and time; both must see the whole-job
totals (sum of units, slowest time), and the sweep shards must cover every
box exactly once. No GPU is involved.
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


def _rank_main(rank, world_size, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    from paper_0910_3915_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        ws, r, local = replicas.world()
        assert (ws, r, local) == (world_size, rank, rank)
        replicas.barrier()
        units, secs = replicas.whole_job(1000.0 * (rank + 1), 2.0 + rank)
        mine = replicas.shard(range(64), rank, world_size)
        got = [None] * world_size
        dist.all_gather_object(got, mine)
        out[rank] = (units, secs, sorted(x for g in got for x in g))
    finally:
        dist.destroy_process_group()


def test_whole_job_totals_and_shards_world_size_2():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        units, secs, boxes = res[rank]
        assert units == 3000.0 and secs == 3.0
        assert boxes == list(range(64))


def test_single_process_is_its_own_job():
    from paper_0910_3915_gb300 import replicas
    assert replicas.whole_job(5.0, 1.5) == (5.0, 1.5)
    assert replicas.shard(range(5), 1, 2) == [1, 3]
    with pytest.raises(ValueError):
        replicas.shard(range(5), 2, 2)
