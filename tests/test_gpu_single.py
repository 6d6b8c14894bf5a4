"""The single-constraint form (PDBO-s: one dual per restart, SBO_OPT_DUAL = 1) on every kernel that
offers it, against the FP64 oracle's ``gda_step_single`` on the same seeded inputs.

Window: 50 iterations with beta scaled down by n, so mu stays positive and the perturbation branch
cannot fire (the same branch-free window as the coordinate form's parity tests).  Tolerances
(normwise per restart): x as for the coordinate form (1e-5 FP32, 2e-2 BF16 / E4M3); mu 1e-4 with
FP32 operands (the dual step adds up n FP32 values of g) and 2e-2 otherwise.  With beta = 0 the
single form must reproduce the coordinate form bit for bit (mu = y_i = ybar throughout)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib
from _helpers import gpu_trajectory, normwise, to_gda_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()
    S.lib()


def _oracle_single(A, cp, p, steps, X0=None):
    if X0 is None:
        X0, _ = O.init_state(A.shape[0], p.restarts, p.seed, p.ybar)
    X = np.array(X0, dtype=np.float64)
    MU = np.full(p.restarts, float(p.ybar))
    xs, mus = [X], [MU]
    for _ in range(steps):
        X, MU, _ = O.gda_step_single(A, cp, X, MU, p.alpha, p.beta, p.delta, p.grad_tol)
        xs.append(X)
        mus.append(MU)
    return np.array(xs), np.array(mus)


def _dense_case(n, B, prec, kernel, tile=0):
    Q, c = W.dense_qubo(n, seed=n + 11)
    p = W.dense_params(Q, restarts=B, iters=200, eval_every=10, seed=3)
    p.beta = p.beta / n
    P = S.Problem.dense(Q, c, precision=prec)
    P.set_option(S.SBO_OPT_KERNEL, kernel)
    if tile:
        P.set_option(S.SBO_OPT_TILE_N, tile)
    return Q, c, p, P


@pytest.mark.parametrize("n,B,prec,kernel,tile,tol", [
    (300, 70, S.SBO_FP32, S.KERNEL_SIMT, 0, 1e-5),
    (40, 33, S.SBO_FP32, S.KERNEL_SIMT, 0, 1e-5),
    (333, 129, S.SBO_BF16, S.KERNEL_TC, 128, 2e-2),
    (600, 300, S.SBO_BF16, S.KERNEL_TC, 512, 2e-2),
    (1000, 256, S.SBO_BF16, S.KERNEL_TC, 1256, 2e-2),
    (1003, 200, S.SBO_BF16, S.KERNEL_TC, 1256, 2e-2),
    (1003, 200, S.SBO_BF16, S.KERNEL_TC, 2256, 2e-2),
])
def test_single_dual_dense_parity(n, B, prec, kernel, tile, tol):
    Q, c, p, P = _dense_case(n, B, prec, kernel, tile)
    with P:
        P.set_option(S.SBO_OPT_DUAL, S.DUAL_SINGLE)
        prm = to_gda_params(p)
        gx, gy = gpu_trajectory(P, prm, 50)
        if tile:
            assert P.info()["tile_n"] == tile
        A, cp = O.canonicalize(Q, c)
        ox, omu = _oracle_single(A, cp, p, 50)
        assert normwise(gx, ox).max() <= tol
        assert np.all(gy == gy[:, :, :1])                   # one dual per restart, broadcast
        mu_tol = 1e-4 if prec == S.SBO_FP32 else 2e-2
        assert normwise(gy[:, :, 0].T, omu.T).max() <= mu_tol
        assert np.all(np.diff(gy[:, :, 0], axis=0) <= 0.0)   # the dual never rises
        P.start(prm)
        P.run(50)                                           # graph replay: the same iterates
        X, Y = P.state()
        assert np.array_equal(X, gx[50]) and np.array_equal(Y, gy[50])


@pytest.mark.parametrize("prec,tol", [(S.SBO_FP32, 1e-5), (S.SBO_BF16, 2e-2), (S.SBO_FP8_E4M3, 2e-2)])
def test_single_dual_csr_parity(prec, tol):
    """Max-Cut on Erdos-Renyi n = 2000 (B = 200, ragged against 128-restart chunks)."""
    n = 2000
    i, j, w = W.maxcut_er(n, 6.0, seed=5)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=200, iters=200, eval_every=10, seed=2)
    p.beta = p.beta / n
    prm = to_gda_params(p)
    with S.Problem.csr(n, rowptr, col, val, c, precision=prec) as P:
        P.set_option(S.SBO_OPT_DUAL, S.DUAL_SINGLE)
        gx, gy = gpu_trajectory(P, prm, 50)
        A, cp = O.canonicalize_csr(n, rowptr, col, val, c)
        ox, omu = _oracle_single(A, cp, p, 50)
        assert normwise(gx, ox).max() <= tol
        mu_tol = 1e-4 if prec == S.SBO_FP32 else 2e-2
        assert normwise(gy[:, :, 0].T, omu.T).max() <= mu_tol
        P.start(prm)
        P.run(50)
        X, Y = P.state()
        assert np.array_equal(X, gx[50]) and np.array_equal(Y, gy[50])


@pytest.mark.parametrize("case", ["simt", "tc", "csr"])
def test_single_dual_with_beta_zero_is_the_coordinate_form_bit_for_bit(case):
    if case == "csr":
        n = 1500
        i, j, w = W.maxcut_er(n, 6.0, seed=1)
        rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
        p = W.graph_params("maxcut", restarts=130, iters=100, eval_every=10, seed=4)
        make = lambda: S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_BF16)
    else:
        n = 500
        Q, c = W.dense_qubo(n, seed=9)
        p = W.dense_params(Q, restarts=100, iters=100, eval_every=10, seed=4)
        prec = S.SBO_FP32 if case == "simt" else S.SBO_BF16
        make = lambda: S.Problem.dense(Q, c, precision=prec)
    p.beta = 0.0
    prm = to_gda_params(p)
    out = []
    for dual in (S.DUAL_COORDINATE, S.DUAL_SINGLE):
        with make() as P:
            P.set_option(S.SBO_OPT_DUAL, dual)
            P.start(prm)
            P.run(100)
            X, Y = P.state()
            out.append((X, Y, P.restart_best(), P.trace()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert all(np.array_equal(a, b) for a, b in zip(out[0][2], out[1][2]))
    assert np.array_equal(out[0][3], out[1][3])


def test_single_dual_paper_steps_reach_binary_points_with_exact_objectives():
    """Torus 40 x 40 with the paper's literal graph parameters (beta = 0.025, unscaled): the single
    dual falls by up to n beta / 4 per step, the iterates become binary quickly, and every best
    record is the exact objective of its own bits."""
    i, j, w = W.maxcut_torus(40, 40, seed=3)
    n = 1600
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    p = W.graph_params("maxcut", restarts=64, iters=300, eval_every=10, seed=1)
    with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P:
        P.set_option(S.SBO_OPT_DUAL, S.DUAL_SINGLE)
        P.gda(to_gda_params(p))
        X, Y = P.state()
        x_star, F_star, t_star, r_star = P.best()
        Fr, tr = P.restart_best()
    assert np.mean((X == 0.0) | (X == 1.0)) > 0.99
    assert np.all(Y[:, 0] < p.ybar)
    assert F_star == -int(np.sum(w * (x_star[i] != x_star[j])))
    assert F_star == Fr.min()


def test_single_dual_is_rejected_where_unsupported():
    Q, c = W.dense_qubo(30, seed=1)
    with S.Problem.dense(Q, c, precision=S.SBO_FP32) as P:
        P.set_option(S.SBO_OPT_DUAL, S.DUAL_SINGLE)
        P.set_option(S.SBO_OPT_KERNEL, S.KERNEL_TINY)
        with pytest.raises(S.SboError):
            P.start(S.params(restarts=4, iters=10, alpha=0.01, beta=0.01, ybar=1.0))
        P.set_option(S.SBO_OPT_KERNEL, 0)
        P.start(S.params(restarts=4, iters=10, alpha=0.01, beta=0.01, ybar=1.0))
        assert P.info()["kernel"] == S.KERNEL_SIMT          # n <= 64 goes to SIMT in this form
