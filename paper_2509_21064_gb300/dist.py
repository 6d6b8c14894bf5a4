"""Multi-process runs: restarts are independent (section 4.2: B initial points, best retained), so
ranks run disjoint sets of restarts with no exchange inside the iteration loop.  The one exchange
is the choice of the global best once the ranks are done: the lexicographic minimum of
(F, t, rank, restart) over every rank's own best, and that rank's candidate bits.

Works with any torch.distributed backend (NCCL across GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def global_best(F: int, t: int, r: int, x: np.ndarray, device=None):
    """Every rank passes its own best (F, t, restart r, bits x); every rank gets back
    (F, t, winning rank, r, x of the winner)."""
    device = device if device is not None else torch.device("cpu")
    rank = dist.get_rank()
    world = dist.get_world_size()
    mine = torch.tensor([int(F), int(t), rank, int(r)], dtype=torch.int64, device=device)
    allv = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(allv, mine)
    rows = sorted(tuple(int(v) for v in a.cpu().tolist()) for a in allv)
    Fw, tw, kw, rw = rows[0]
    bits = torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint8)).to(device)
    dist.broadcast(bits, src=kw)
    return Fw, tw, kw, rw, bits.cpu().numpy()


def max_over_ranks(values, device=None):
    """Element-wise maximum of a list of floats over all ranks (slowest-rank timing)."""
    device = device if device is not None else torch.device("cpu")
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu().tolist()]
