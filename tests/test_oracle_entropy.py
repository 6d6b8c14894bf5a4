"""Pins of the oracle's entropy constraint function (section 3.1 names x log x + (1-x) log(1-x)
among the choices of g and lists the conditions g must meet)."""
import numpy as np

import oracle as O
import workloads as W


def test_entropy_meets_the_conditions_of_section_3_1():
    x = np.linspace(0.0, 1.0, 2001)
    gx = O.g_entropy(x)
    assert gx[0] == 0.0 and gx[-1] == 0.0                       # g(0) = g(1) = 0 (continuous extension)
    assert np.all(gx[1:-1] < 0.0)                                # negative inside
    assert np.allclose(gx, O.g_entropy(1.0 - x), atol=1e-15)     # symmetric
    assert np.all(np.diff(gx, 2) >= -1e-15)                      # convex
    assert abs(O.g_entropy(0.5) + np.log(2.0)) <= 1e-15          # g(1/2) = -ln 2
    gp = O.g_entropy_prime(x[1:-1])
    assert O.g_entropy_prime(0.5) == 0.0
    assert np.all(gp[x[1:-1] < 0.5] < 0.0) and np.all(gp[x[1:-1] > 0.5] > 0.0)


def test_entropy_derivative_is_the_central_difference_and_is_clamped_at_the_ends():
    x = np.linspace(0.01, 0.99, 99)
    h = 1e-7
    fd = (O.g_entropy(x + h) - O.g_entropy(x - h)) / (2 * h)
    assert np.allclose(O.g_entropy_prime(x), fd, rtol=1e-6, atol=1e-7)
    eps = O.ENTROPY_EPS
    assert O.g_entropy_prime(0.0) == O.g_entropy_prime(eps) < -13.0
    assert O.g_entropy_prime(1.0) == O.g_entropy_prime(1.0 - eps) > 13.0


def test_entropy_lagrangian_gradient_and_binary_points():
    Q, c = W.dense_qubo(12, seed=3)
    A, cp = O.canonicalize(Q, c)
    rng = np.random.default_rng(2)
    X = rng.uniform(0.05, 0.95, size=(2, 12))
    Y = rng.normal(scale=5.0, size=(2, 12))
    L, GX, GY = O.lagrangian(A, cp, X, Y, "entropy")
    h = 1e-6
    for r, k in ((0, 0), (1, 7), (0, 11)):
        E = np.zeros_like(X)
        E[r, k] = h
        fd = (O.lagrangian(A, cp, X + E, Y, "entropy")[0][r] - O.lagrangian(A, cp, X - E, Y, "entropy")[0][r]) / (2 * h)
        assert abs(fd - GX[r, k]) <= 1e-6 * max(1.0, abs(GX[r, k]))
    assert np.array_equal(GY, O.g_entropy(X))
    Bits = rng.integers(0, 2, size=(4, 12))
    Lb, _, _ = O.lagrangian(A, cp, Bits.astype(np.float64), rng.normal(size=(4, 12)) * 30, "entropy")
    assert np.array_equal(Lb, O.objective_batch(Q, c, Bits).astype(np.float64))


def test_entropy_run_keeps_the_box_and_a_falling_dual():
    Q, c = W.dense_qubo(30, seed=8)
    p = W.dense_params(Q, restarts=5, iters=80, eval_every=10, seed=1)
    out = O.run(Q, c, p.restarts, 80, p.alpha, p.beta, p.ybar, p.delta, p.grad_tol, 10, p.seed,
                dump_iters=80, gkind="entropy")
    xs, ys = np.array(out["dumps"]["x"]), np.array(out["dumps"]["y"])
    assert np.all((xs >= 0.0) & (xs <= 1.0))
    dy = np.diff(ys, axis=0)
    assert np.all(dy <= 0.0) and np.all(dy >= -p.beta * np.log(2.0) - 1e-12)
    assert out["F_star"] == O.objective(Q, c, out["x_star"])
