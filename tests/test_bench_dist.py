"""Replica sharding of bench.py on CPU: two gloo ranks take disjoint job ids and the timing
reduction returns the maximum over ranks (no data-path collective exists)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import sys
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    d = bench.Dist()
    try:
        ids = list(bench.shard(100, d.rank))
        d.barrier()
        m = d.max(float(10 + rank))
        q.put((rank, ids, m, d.world))
    finally:
        d.close()


def test_two_gloo_ranks_shard_and_reduce():
    if torch.cuda.is_available():
        pytest.skip("exercises the CPU (gloo) path")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, ids0, m0, w0), (r1, ids1, m1, w1) = res
    assert w0 == w1 == 2
    assert ids0 == list(range(0, 100)) and ids1 == list(range(100, 200))  # weak scaling: disjoint shards
    assert m0 == m1 == 11.0  # max over ranks
