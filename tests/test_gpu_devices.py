"""Function attributes and occupancy answers belong to the context of the device that was current
when they were set, so the library sets and caches them per device: tensor-core problems on two
GPUs in one process run, and give the same results on both (skipped with fewer than two GPUs)."""
import pytest

import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib

pytestmark = pytest.mark.gpu


def test_tensor_core_problems_on_two_devices_in_one_process():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    build_lib()
    Q, c = W.dense_qubo(600, seed=4)
    p = W.dense_params(Q, restarts=300, iters=20, eval_every=10, seed=2)
    best = {}
    for dev in (0, 1):
        torch.cuda.set_device(dev)
        for tile in (256, 512, 1128):      # single CTA, CTA pairs, cluster split-K
            with S.Problem.dense(Q, c, precision=S.SBO_BF16) as P:
                P.set_option(S.SBO_OPT_TILE_N, tile)
                P.gda(S.params(**p.asdict()))
                best[(dev, tile)] = P.best()[1]
    torch.cuda.set_device(0)
    for tile in (256, 512, 1128):
        assert best[(0, tile)] == best[(1, tile)], best
