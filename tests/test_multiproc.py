"""The multi-rank host logic of bench.py on CPU with the gloo backend, two
ranks: independent work items are sharded without overlap or loss, and the
timing taken is the slowest rank's (one all-reduce, no data-path collective)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import meshgen as mg
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env() == (rank, world, rank)
        specs = mg.batch_instances()
        mine = bench.shard(specs, rank, world)
        # every rank reports its share's (kind, mesh, alpha) keys and a fake time
        keys = [(s["kind"], s["mesh"], s["alpha"]) for s in mine]
        gathered = [None] * world
        dist.all_gather_object(gathered, keys)
        t = bench.max_over_ranks(1.0 + rank, world, "cpu")
        out[rank] = {"keys": gathered, "tmax": t, "n": len(specs)}
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_slowest_rank_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r = res[rank]
        flat = [k for part in r["keys"] for k in part]
        assert len(flat) == r["n"] == 48                    # nothing lost
        assert len(set(flat)) == 48                         # no instance on two ranks
        assert abs(len(r["keys"][0]) - len(r["keys"][1])) <= 1  # balanced
        assert r["tmax"] == 2.0                             # the slowest rank's time
