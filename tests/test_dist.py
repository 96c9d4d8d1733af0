"""The multi-rank path of the benchmark on CPU (gloo, world size 2): max-over-ranks time,
summed work, disjoint frame blocks.  No GPU involved."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1407_2074_b300 import dist as D

    t, w = D.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1))
    dist.barrier()
    out[rank] = (t, w, D.frames_for_rank(rank, 4, 60))
    dist.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        t, w, frames = out[r]
        assert t == 15.0 and w == 300.0
    assert set(out[0][2]).isdisjoint(out[1][2])


def test_single_process_aggregation_is_identity():
    from paper_1407_2074_b300 import dist as D

    assert D.aggregate(3.5, 7.0) == (3.5, 7.0)
    assert D.env()[0] >= 1


def test_frames_disjoint_until_the_orbit_wraps():
    from paper_1407_2074_b300 import dist as D

    for ranks, steps in ((2, 30), (4, 15), (8, 7)):  # ranks x steps <= 60: disjoint
        sets = [set(D.frames_for_rank(r, steps, 60)) for r in range(ranks)]
        assert sum(len(s) for s in sets) == len(set().union(*sets)) == ranks * steps
    # 8 ranks x 23 steps (3 warm-up + 20 timed) > 60: the orbit wraps and views repeat
    frames = [D.frames_for_rank(r, 23, 60) for r in range(8)]
    assert all(len(f) == 23 and all(0 <= x < 60 for x in f) for f in frames)
    assert len(set().union(*map(set, frames))) == 60
