"""Deferred evaluation of sparse runs replayed from CUDA graphs: a replayed block leaves the
candidates of its last iteration pending, and the next block evaluates them on a graph branch
beside its first K - 1 steps; every call that reads results evaluates what is pending first.
Against the same run without graphs (every evaluation right after its step): identical states,
per-restart bests, min-F traces and global bests, for several splittings of the run into calls,
with and without results read between the calls, K even and odd, T not a multiple of K."""
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


def _run(n, csr, prec, prm, graph, chunks, peek, eval_mode=S.EVAL_MODE_RULE):
    rowptr, col, val, c = csr
    seen = []
    with S.Problem.csr(n, rowptr, col, val, c, precision=prec) as P:
        P.set_option(S.SBO_OPT_USE_GRAPH, int(graph))
        P.set_option(S.SBO_OPT_EVAL_MODE, eval_mode)
        P.start(prm)
        for k in chunks:
            P.run(k)
            if peek:   # results between calls: pending evaluations are flushed here
                Fr, tr = P.restart_best()
                seen.append((Fr.copy(), tr.copy(), P.trace().copy()))
        P.sync()
        X, Y = P.state()
        Fr, tr = P.restart_best()
        best = P.best()
        trace = P.trace()
    return X, Y, Fr, tr, best, trace, seen


def _same(a, b):
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)
    assert a[4][1:] == b[4][1:] and np.array_equal(a[4][0], b[4][0])
    assert np.array_equal(a[5], b[5])
    assert len(a[6]) == len(b[6])
    for (f1, t1, s1), (f2, t2, s2) in zip(a[6], b[6]):
        assert np.array_equal(f1, f2) and np.array_equal(t1, t2) and np.array_equal(s1, s2)


@pytest.mark.parametrize("K,T,chunks", [(7, 100, (100,)), (7, 100, (3, 11, 1, 28, 57)), (10, 120, (10,) * 12),
                                         (2, 31, (5, 4, 22)), (10, 95, (40, 40, 15))])
@pytest.mark.parametrize("peek", [False, True])
@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_BF16])
@pytest.mark.parametrize("mode", [S.EVAL_MODE_RULE, S.EVAL_MODE_INLINE])
def test_deferred_evaluations_match_immediate_ones(K, T, chunks, peek, prec, mode):
    """Erdos-Renyi n = 3001, B = 200 (ragged rows and restart chunks)."""
    n = 3001
    i, j, w = W.maxcut_er(n, 6.0, seed=3)
    csr = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=200, iters=T, eval_every=K, seed=5)
    prm = to_gda_params(p)
    a = _run(n, csr, prec, prm, 1, chunks, peek, mode)
    b = _run(n, csr, prec, prm, 0, chunks, peek)
    _same(a, b)
    x_star, F_star = a[4][0], a[4][1]
    assert F_star == -int(np.sum(w * (x_star[i] != x_star[j])))
    assert len(a[5]) == len(range(K, T + 1, K)) + (T % K != 0)   # one trace entry per evaluation


def test_deferred_evaluations_on_the_torus_with_two_restart_groups_per_warp():
    """100 x 100 torus, B = 512 (256 restarts per warp in the update and the evaluation), K = 10,
    the run split into calls of one block each (as the benchmark drives it)."""
    i, j, w = W.maxcut_torus(100, 100, seed=0)
    n = 10000
    csr = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=512, iters=80, eval_every=10, seed=2)
    prm = to_gda_params(p)
    a = _run(n, csr, S.SBO_FP32, prm, 1, (10,) * 8, False)
    b = _run(n, csr, S.SBO_FP32, prm, 0, (10,) * 8, False)
    _same(a, b)


@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_FP8_E4M3])
def test_deferred_evaluations_on_the_regular_graph(prec):
    """Random 4-regular graph, n = 20,000, B = 512: x and y overflow L2 (the streaming update
    forms), the evaluations run beside the next block; the run split into blocks of one evaluation
    each (as the benchmark drives it) gives what in-line evaluation gives."""
    n = 20000
    i, j, w = W.maxcut_regular(n, 4, seed=0)
    csr = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=512, iters=70, eval_every=10, seed=2)
    prm = to_gda_params(p)
    a = _run(n, csr, prec, prm, 1, (10,) * 7, False)    # no reads between calls: nothing flushes
    b = _run(n, csr, prec, prm, 0, (10,) * 7, False)
    _same(a, b)


@pytest.mark.parametrize("peek", [False, True])
def test_deferred_evaluations_of_max3cut(peek):
    """Max-3-Cut of a 30 x 40 +-1 torus, B = 100, K = 7, T = 60, the run split at points that are
    and are not evaluation points: parts, cuts, traces and states as with in-line evaluation."""
    i, j, w = W.maxcut_torus(30, 40, seed=1)
    n = 1200
    p = W.GdaParams(restarts=100, iters=60, alpha=0.01, beta=0.01, ybar=6.0, eval_every=7, seed=4)
    prm = to_gda_params(p)
    out = []
    for graph in (1, 0):
        seen = []
        with S.Problem.maxkcut(n, i, j, w, 3) as P:
            P.set_option(S.SBO_OPT_USE_GRAPH, graph)
            P.start(prm)
            for k in (3, 11, 1, 28, 17):
                P.run(k)
                if peek:
                    Fr, tr = P.restart_best()
                    seen.append((Fr.copy(), tr.copy(), P.trace().copy()))
            P.sync()
            X, Y = P.state()
            Fr, tr = P.restart_best()
            out.append((X, Y, Fr, tr, P.best(), P.trace(), seen))
    _same(out[0], out[1])
    parts, F = out[0][4][0], out[0][4][1]
    assert F == -int(np.sum(w * (parts[i] != parts[j])))


def test_graphs_switched_off_and_on_between_calls():
    """Replay switched off while an evaluation is pending, then on again: the pending evaluation
    runs in line and nothing is lost or evaluated twice."""
    n = 3001
    i, j, w = W.maxcut_er(n, 6.0, seed=3)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=200, iters=120, eval_every=10, seed=5)
    prm = to_gda_params(p)
    out = []
    for toggle in (True, False):
        with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P:
            P.set_option(S.SBO_OPT_USE_GRAPH, 1 if toggle else 0)
            P.start(prm)
            for k, g in ((40, 0), (30, 1), (50, 1)):
                P.run(k)
                if toggle:
                    P.set_option(S.SBO_OPT_USE_GRAPH, g)
            P.sync()
            X, Y = P.state()
            Fr, tr = P.restart_best()
            out.append((X, Y, Fr, tr, P.best(), P.trace(), []))
    _same(out[0], out[1])
    assert len(out[0][5]) == 12
