"""Programmatic dependent launch of the sparse kernel (each iteration's launch overlaps the previous
iteration; every kernel waits for its predecessor's writes before reading them) against plain
stream order: states, per-restart bests, the min-F trace and the global best are identical, with
and without CUDA-graph replay, on every operand type."""
import numpy as np
import pytest

import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib
from _helpers import to_gda_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()
    S.lib()


def _run(rowptr, col, val, c, n, prec, prm, pdl, graph, chunks):
    with S.Problem.csr(n, rowptr, col, val, c, precision=prec) as P:
        P.set_option(S.SBO_OPT_PDL, int(pdl))
        P.set_option(S.SBO_OPT_USE_GRAPH, int(graph))
        P.start(prm)
        for k in chunks:
            P.run(k)
        P.sync()
        X, Y = P.state()
        Fr, tr = P.restart_best()
        best = P.best()
        trace = P.trace()
    return X, Y, Fr, tr, best, trace


@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_BF16, S.SBO_FP8_E4M3])
@pytest.mark.parametrize("graph", [0, 1])
def test_dependent_launches_are_bit_identical_to_stream_order(prec, graph):
    """Erdos-Renyi n = 3001 (ragged against the 8 rows of a block), B = 200 (ragged against the
    128-restart chunks), K = 7 (odd: the operand buffer parity flips per block); runs split at
    points that are and are not evaluation points."""
    n = 3001
    i, j, w = W.maxcut_er(n, 6.0, seed=3)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=200, iters=100, eval_every=7, seed=5)
    prm = to_gda_params(p)
    chunks = (3, 11, 1, 28, 57)
    a = _run(rowptr, col, val, c, n, prec, prm, 1, graph, chunks)
    b = _run(rowptr, col, val, c, n, prec, prm, 0, graph, chunks)
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)
    assert a[4][1:] == b[4][1:] and np.array_equal(a[4][0], b[4][0])
    assert np.array_equal(a[5], b[5])
    x_star, F_star = a[4][0], a[4][1]
    assert F_star == -int(np.sum(w * (x_star[i] != x_star[j])))
