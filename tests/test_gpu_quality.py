"""Solution quality of the chosen form against the plain FP32 form at equal iterations: the BF16
tensor-core contraction (x rounded to BF16 before it, FP32 accumulation and master iterates) and
the FP32 CUDA-core contraction run the same T iterations from the same x^0; their best objectives
agree within 0.1 % (the mixed-precision error changes trajectories, not the quality reached)."""
import numpy as np
import pytest

import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib
from _helpers import to_gda_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,B,T", [(5000, 256, 300), (2000, 256, 400)])
def test_best_objective_within_a_thousandth_of_the_fp32_form(n, B, T):
    build_lib()
    Q, c = W.dense_qubo(n, seed=1)
    p = W.dense_params(Q, restarts=B, iters=T, eval_every=50, seed=3)
    best = {}
    for prec in (S.SBO_BF16, S.SBO_FP32):
        with S.Problem.dense(Q, c, precision=prec) as P:
            if prec == S.SBO_FP32:
                P.set_option(S.SBO_OPT_KERNEL, S.KERNEL_SIMT)
            P.gda(to_gda_params(p))
            best[prec] = int(P.best()[1])
    gap = abs(best[S.SBO_BF16] - best[S.SBO_FP32]) / abs(best[S.SBO_FP32])
    print(n, B, T, best, gap)
    assert gap <= 1e-3
