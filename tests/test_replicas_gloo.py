"""The multi-rank path (replicas, barrier, max/sum over ranks) with two gloo ranks on CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_1201_3185_gb300.replicas import Replicas
    rep = Replicas.from_env(backend="gloo")
    rep.barrier()
    elapsed = 1.0 + rank  # rank-dependent "timings"
    m = rep.max(elapsed)
    tot = rep.total(10.0 * (rank + 1))
    seed = rep.replica_seed(1)
    rep.barrier()
    rep.close()
    out.put((rank, m, tot, seed))


def test_two_gloo_ranks():
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
    assert [r[1] for r in res] == [2.0, 2.0]   # max over ranks seen by every rank
    assert [r[2] for r in res] == [30.0, 30.0]  # sum over ranks
    assert res[0][3] != res[1][3]               # independent replicas


def test_single_rank_needs_no_group(monkeypatch):
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    from paper_1201_3185_gb300.replicas import Replicas
    rep = Replicas.from_env(backend="gloo")
    assert rep.world_size == 1 and rep.max(3.5) == 3.5 and rep.total(2.0) == 2.0
