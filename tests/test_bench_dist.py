"""The benchmark's multi-rank host logic on CPU: two gloo ranks (no GPU).

Under torchrun every rank answers its own shard of the query stream against a
replicated dictionary; the process group carries only the barrier and the
max-over-ranks time.  These tests run that logic with world_size 2 on the
gloo backend: the rank setup from the environment, the max over ranks, and
the per-rank query shards (same size and length mix, distinct, reproducible).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import bench
    import datagen
    args = bench.parse(["--gpus", str(world)])
    w_, r_, l_, pg = bench.dist_setup(args)
    bench.barrier(pg)
    t = bench.max_over_ranks(pg, 1.5 + rank)  # each rank's "time"
    w = datagen.english1m(3000, 200)
    qs = bench.rank_queries(w, rank)
    digest = {m: (len(q), int(q.chars.astype(np.int64).sum()), q.lengths().tolist()[:5]) for m, q in qs.items()}
    bench.barrier(pg)
    pg.destroy_process_group()
    out.put((rank, w_, r_, t, digest))


@pytest.mark.timeout(300)
def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, rk0, t0, d0), (r1, w1, rk1, t1, d1) = res
    assert (w0, w1) == (2, 2) and (rk0, rk1) == (0, 1)
    assert t0 == t1 == 2.5  # the max over ranks, seen by both
    for m in ("ham", "lev"):
        assert d0[m][0] == d1[m][0] == 200  # same shard size
        assert d0[m][1] != d1[m][1]  # distinct patterns
    # reproducible: rank 1's shard is the same in a fresh process
    sys.path.insert(0, ROOT)
    import bench
    import datagen
    w = datagen.english1m(3000, 200)
    again = bench.rank_queries(w, 1)
    for m in ("ham", "lev"):
        assert int(again[m].chars.astype(np.int64).sum()) == d1[m][1]
