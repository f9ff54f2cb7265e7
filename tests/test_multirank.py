"""Multi-rank host logic of the benchmark on CPU: world_size 2 over gloo.

Each rank reports a different time; every rank must see the maximum, the
barrier must hold, and the replicas must simulate distinct seeded scenes."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2402_01181_gb300 import dist as D
    from paper_2402_01181_gb300 import scenes
    r = D.Ranks(backend="gloo")
    r.barrier()
    m = r.max(10.0 + 5.0 * rank)
    x = scenes.cube8k(seed=D.replica_seed(rank)).x
    r.barrier()
    r.close()
    out.put((rank, m, float(x[:, 0].sum())))


def test_max_over_ranks_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [m for _, m, _ in res] == [15.0, 15.0]
    assert res[0][2] != res[1][2]        # distinct replicas


def test_single_rank_is_a_no_op(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2402_01181_gb300 import dist as D
    r = D.Ranks()
    r.barrier()
    assert r.max(3.5) == 3.5
    r.close()
