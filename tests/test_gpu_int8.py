"""sbo_create_dense_i8: an int8 Q builds the same canonical problem as its int32 copy (diagonal
and negative entries included): identical iterates, bests and evaluations on both precisions."""
import numpy as np
import pytest

import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib
from _helpers import to_gda_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_BF16])
def test_int8_and_int32_inputs_give_the_same_run(prec):
    build_lib()
    n = 777
    rng = np.random.default_rng(3)
    M = rng.integers(-128, 128, size=(n, n)).astype(np.int32)   # not symmetric, full int8 range
    c = rng.integers(-1000, 1000, size=n).astype(np.int32)
    p = W.dense_params(M, restarts=100, iters=60, eval_every=10, seed=2)
    prm = to_gda_params(p)
    out = []
    for Q in (M, M.astype(np.int8)):
        with S.Problem.dense(Q, c, precision=prec) as P:
            P.start(prm)
            P.run(60)
            X, Y = P.state()
            bits = rng.integers(0, 2, size=(5, n)).astype(np.uint8) if not out else out[0][3]
            out.append((X, Y, P.best(), bits, S.sbo_eval(P.h, bits)))
    (X1, Y1, b1, _, F1), (X2, Y2, b2, _, F2) = out
    assert np.array_equal(X1, X2) and np.array_equal(Y1, Y2)
    assert np.array_equal(b1[0], b2[0]) and b1[1:] == b2[1:]
    assert np.array_equal(F1, F2)
