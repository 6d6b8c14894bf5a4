"""Pins of the oracle's dual certificate (the paper's section on the dual certificate)."""
import numpy as np
import scipy.optimize as so

import oracle as O
import workloads as W


def _convex_ybar(A):
    lam = float(np.linalg.eigvalsh(A).min())
    return max(0.0, -lam / 2.0) + 1e-6      # A + 2 ybar I is positive semidefinite


def _box_min(A, cp, ybar):
    n = A.shape[0]
    fun = lambda x: float(O.lagrangian(A, cp, x[None, :], np.full((1, n), ybar))[0][0])
    jac = lambda x: O.lagrangian(A, cp, x[None, :], np.full((1, n), ybar))[1][0]
    res = so.minimize(fun, np.full(n, 0.5), jac=jac, method="L-BFGS-B", bounds=[(0.0, 1.0)] * n,
                      options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    return res.x, res.fun


def test_certificate_is_tight_at_the_box_minimiser_and_below_it_elsewhere():
    Q, c = W.dense_qubo(14, seed=6)
    A, cp = O.canonicalize(Q, c)
    ybar = _convex_ybar(A)
    xs, Ls = _box_min(A, cp, ybar)
    assert abs(O.certificate(A, cp, ybar, xs) - Ls) <= 1e-6 * max(1.0, abs(Ls))
    rng = np.random.default_rng(0)
    for _ in range(20):
        assert O.certificate(A, cp, ybar, rng.random(14)) <= Ls + 1e-9


def test_certificate_is_a_lower_bound_on_the_brute_force_minimum():
    for seed in range(4):
        Q, c = W.dense_qubo(16, seed=20 + seed)
        A, cp = O.canonicalize(Q, c)
        ybar = _convex_ybar(A)
        Fmin, _ = O.brute_force(Q, c)
        rng = np.random.default_rng(seed)
        for x in (np.full(16, 0.5), rng.random(16), _box_min(A, cp, ybar)[0]):
            assert O.certificate(A, cp, ybar, x) <= Fmin
