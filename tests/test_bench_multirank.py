"""Host logic of bench.py for N > 1 replicas, on CPU with the gloo backend
(world size 2): the job time is the slowest rank's, the regions are summed,
and only rank 0 prints."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_setup()
    t, n = bench.aggregate_over_ranks(1.5 + rank, 1000 * (rank + 1), ws, "cpu")
    q.put((r, ws, local, t, n))
    dist.destroy_process_group()


def test_two_replicas_aggregate_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, ws, local, t, n) in enumerate(out):
        assert (r, ws, local) == (rank, 2, rank)
        assert t == 2.5  # the slowest rank
        assert n == 3000.0  # regions of both ranks


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_over_ranks(2.0, 7, 1) == (2.0, 7.0)
