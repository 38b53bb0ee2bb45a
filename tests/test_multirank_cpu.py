"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): ranks own
disjoint phantoms that together cover all of them, and the reported time is
the maximum over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.rank_phantoms(rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    slowest = bench.max_over_ranks(1.5 + rank, dist)
    dist.destroy_process_group()
    q.put((rank, gathered, slowest))


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_split_phantoms_and_report_the_slowest(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    for rank, gathered, slowest in out:
        flat = [x for part in gathered for x in part]
        assert sorted(flat) == list(range(bench.N_PHANTOMS))      # covering
        assert len(flat) == len(set(flat))                          # disjoint
        assert slowest == 1.5 + (world - 1)                         # max over ranks


def test_more_ranks_than_phantoms_still_get_work():
    import bench
    assert bench.rank_phantoms(12, 16) == [2]
