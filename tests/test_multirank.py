"""Replica host logic of bench.py on two gloo ranks (CPU): every rank joins the
process group, the barrier completes, and the elapsed time reported is the
maximum over ranks.  The sort itself has no data-path collective (one grid
does not shard; N GPUs run N independent replicas)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    w, r, local, pg = bench._dist_setup()
    assert pg is not None and w == world and r == rank
    v = bench._max_over_ranks(float(10 * (rank + 1)), pg, "cpu")
    bench._barrier(pg)
    q.put((rank, v))
    pg.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert got == [(r, 10.0 * world) for r in range(world)]
