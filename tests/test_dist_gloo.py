"""The multi-process path on CPU (gloo, world size 2): the cross-rank choice of the global best and
the slowest-rank timing that bench.py uses under torchrun."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cases, out):
    import torch.distributed as dist
    from paper_2509_21064_gb300.dist import global_best, max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = []
        for case in cases:
            F, t, r = case[rank]
            x = np.full(6, rank, dtype=np.uint8)
            res.append(global_best(F, t, r, x))
        res.append(max_over_ranks([1.0 + rank, 5.0 - rank]))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_global_best_is_the_lexicographic_minimum_over_ranks(world):
    cases = [
        [(-10, 50, 3), (-12, 900, 0)],     # smaller F wins regardless of t
        [(-12, 100, 7), (-12, 100, 1)],    # equal F and t: lower rank wins
        [(-12, 150, 0), (-12, 100, 9)],    # equal F: earlier t wins
    ]
    expect = [(-12, 900, 1, 0), (-12, 100, 0, 7), (-12, 100, 1, 9)]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, world, port, cases, out)) for k in range(world)]
    for p in procs:
        p.start()
    got = dict(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        res = got[rank]
        for (Fw, tw, kw, rw, xw), e in zip(res[:-1], expect):
            assert (Fw, tw, kw, rw) == e
            assert np.all(xw == kw)        # the winner's bits reach every rank
        assert res[-1] == [2.0, 5.0]
