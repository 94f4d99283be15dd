"""The multi-GPU host path on CPU: two gloo ranks own disjoint event sets of
equal size (weak scaling, no solver data exchanged), the timed region's
barrier completes, and the elapsed time reported is the max over ranks."""
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
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1510_06340_b300 import dist as D
    w, r, lr = D.world()
    ids = D.rank_events(5, r)
    D.barrier()
    t = D.max_over_ranks(1.5 + r)
    q.put((r, w, ids, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_events_and_reduce_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, ids0, t0), (r1, w1, ids1, t1) = out
    assert (w0, w1) == (2, 2)
    assert len(ids0) == len(ids1) == 5 and not set(ids0) & set(ids1)
    assert sorted(ids0 + ids1) == list(range(10))
    assert t0 == t1 == 2.5


def test_single_process_defaults():
    from paper_1510_06340_b300 import dist as D
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert D.world() == (1, 0, 0)
    assert D.max_over_ranks(3.0) == 3.0
