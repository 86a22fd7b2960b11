"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The search shards by gallery block with no data-path collective: each rank
searches its own blocks, and the only cross-rank operations are a barrier and
the max of the per-rank timings.  This checks those two operations and that
ranks draw distinct galleries.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import workloads as W
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    d = bench.Dist(world, "gloo")
    d.barrier()
    got = d.max(float(rank + 1) * 1.5, "cpu")
    feats = W.gallery_features(64, 8, bench.FEAT_SEED + 7919 * rank)
    d.barrier()
    d.close()
    out.put((rank, got, feats.tobytes()))


def test_two_ranks_barrier_and_max():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(abs(v - 3.0) < 1e-12 for _, v, _ in res)   # max over ranks
    assert res[0][2] != res[1][2]                          # distinct per-rank galleries
