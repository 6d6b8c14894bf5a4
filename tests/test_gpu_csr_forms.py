"""Every form of the sparse update kernel (SBO_OPT_CSR_FORM: one row per warp with 128 or 256
restarts, pipelined rows, each of them with or without L2 eviction priorities, the state resident in
shared memory over several iterations per launch, rows staged in shared memory by bulk copies)
computes the same sums in the same order, so all of them give bit-identical runs; the staged form
is also held to the FP64 oracle.  The resident form serves the graphs whose state fits in shared
memory (ER and hubs here; the torus at B = 600 falls back to the rule).  The graphs cover ragged restart chunks (B = 200), two chunks of restarts per row (B = 600,
the second one short), isolated vertices, and hub vertices whose rows span several stages."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib
from _helpers import gpu_trajectory, normwise, oracle_trajectory, to_gda_params

pytestmark = pytest.mark.gpu

FORMS = [S.CSR_FORM_ROW1, S.CSR_FORM_ROW2, S.CSR_FORM_PIPE2, S.CSR_FORM_ROW1_STREAM, S.CSR_FORM_ROW2_STREAM,
         S.CSR_FORM_PIPE2_STREAM, S.CSR_FORM_RESIDENT, S.CSR_FORM_STAGED]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()
    S.lib()


def _hubs(n=3000, seed=5):
    """Sparse random graph with +-1 weights, 40 isolated vertices and 6 hubs of degree ~60."""
    rng = np.random.default_rng(seed)
    i, j, w = W.maxcut_er(n, 4.0, seed=seed)
    iso = set(rng.choice(n, size=40, replace=False).tolist())
    keep = np.array([(a not in iso) and (b not in iso) for a, b in zip(i, j)])
    i, j, w = i[keep], j[keep], w[keep]
    pairs = set(zip(i.tolist(), j.tolist()))
    hubs = [v for v in rng.choice(n, size=12, replace=False).tolist() if v not in iso][:6]
    for h in hubs:
        for v in rng.choice(n, size=60, replace=False).tolist():
            if v != h and v not in iso:
                pairs.add((min(h, v), max(h, v)))
    pairs = sorted(pairs)
    i = np.array([p[0] for p in pairs], np.int32)
    j = np.array([p[1] for p in pairs], np.int32)
    w = np.where(rng.integers(0, 2, size=len(pairs)) == 1, 1, -1).astype(np.int32)
    return n, i, j, w


GRAPHS = {
    "er_b200": (lambda: (2000, *W.maxcut_er(2000, 6.0, seed=3)), 200),
    "torus_b600": (lambda: (10000, *W.maxcut_torus(100, 100, seed=2)), 600),
    "hubs_b130": (_hubs, 130),
}


@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_FP8_E4M3])
@pytest.mark.parametrize("graph", list(GRAPHS))
def test_every_sparse_form_gives_the_same_bits(graph, prec):
    make, B = GRAPHS[graph]
    n, i, j, w = make()
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=B, iters=3000, eval_every=10, seed=1)
    prm = to_gda_params(p)
    runs = []
    for form in FORMS:
        with S.Problem.csr(n, rowptr, col, val, c, precision=prec) as P:
            P.set_option(S.SBO_OPT_CSR_FORM, form)
            gx, gy = gpu_trajectory(P, prm, 12)            # direct launches, one per call
            P.start(prm)
            P.run(30)                                       # graph replay and evaluations
            X, Y = P.state()
            Fr, tr = P.restart_best()
            runs.append((gx, gy, X, Y, Fr, tr))
    for form, r in zip(FORMS[1:], runs[1:]):
        for a, b in zip(runs[0], r):
            assert np.array_equal(a, b), form
    # the staged form against the FP64 oracle
    gx, gy = runs[-1][0], runs[-1][1]
    A, cp = O.canonicalize_csr(n, rowptr, col, val, c)
    ox, oy, _ = oracle_trajectory(None, None, p, 12, A=A, cp=cp)
    tol = 1e-5 if prec == S.SBO_FP32 else 2e-2
    assert normwise(gx, ox).max() <= tol and normwise(gy, oy).max() <= tol


def test_autotuned_form_is_reported_and_kept():
    """The autotuner picks one of the forms at start; the run with it equals the forced form."""
    n, (i, j, w) = 10000, W.maxcut_torus(100, 100, seed=0)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=512, iters=3000, eval_every=10, seed=0)
    prm = to_gda_params(p)
    with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P:
        P.start(prm)
        P.run(20)
        X, Y = P.state()
    with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P:
        P.set_option(S.SBO_OPT_CSR_FORM, S.CSR_FORM_ROW1)
        P.start(prm)
        P.run(20)
        X1, Y1 = P.state()
    assert np.array_equal(X, X1) and np.array_equal(Y, Y1)


def test_resident_form_is_used_where_it_fits_and_keeps_its_bits_across_launch_sizes():
    """The resident form on Max-Cut ER n = 2,000, B = 256 (the benchmark's small graph): reported by
    sbo_info, and the same bits with one launch per iteration, 3 iterations per launch and whole
    blocks per launch, with and without graphs (T = 37 crosses the evaluations at 10, 20, 30)."""
    n = 2000
    i, j, w = W.maxcut_er(n, 6.0, seed=0)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    prm = to_gda_params(W.graph_params("maxcut", restarts=256, iters=3000, eval_every=10, seed=0))
    runs = []
    for per_launch in (1, 3, 0):
        for graph in (0, 1):
            with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P:
                P.set_option(S.SBO_OPT_CSR_FORM, S.CSR_FORM_RESIDENT)
                P.set_option(S.SBO_OPT_STEPS_PER_LAUNCH, per_launch)
                P.set_option(S.SBO_OPT_USE_GRAPH, graph)
                P.start(prm)
                assert P.info()["tile_n"] == S.CSR_FORM_RESIDENT
                P.run(37)
                X, Y = P.state()
                Fr, tr = P.restart_best()
                runs.append((X, Y, Fr, tr, P.trace()))
    with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P:
        P.set_option(S.SBO_OPT_CSR_FORM, S.CSR_FORM_ROW1)
        P.start(prm)
        P.run(37)
        X, Y = P.state()
        Fr, tr = P.restart_best()
        runs.append((X, Y, Fr, tr, P.trace()))
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            assert np.array_equal(a, b)

