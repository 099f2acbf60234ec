"""Multi-process plumbing of the benchmark (one process per GPU) on CPU with
the gloo backend, world size 2: problem sharding gives every item to exactly
one rank, and the max / sum reductions used for the timed region agree across
ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    from paper_2402_12373_gb300 import dist as D
    D.init("gloo")
    r, lr, w = D.env_rank()
    items = list(range(11))
    mine = D.shard(items, r, w)
    t = D.reduce_max(1.5 + r)
    n = D.reduce_sum(len(mine))
    D.barrier()
    q.put((r, mine, t, n))
    dist.destroy_process_group()


def test_shard_and_reductions_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, n0), (r1, m1, t1, n1) = out
    assert sorted(m0 + m1) == list(range(11)) and not set(m0) & set(m1)
    assert t0 == t1 == 2.5
    assert n0 == n1 == 11


def test_shard_rejects_bad_rank():
    from paper_2402_12373_gb300 import dist as D
    with pytest.raises(ValueError):
        D.shard([1, 2], 2, 2)
