"""Pins of the oracle's single-constraint variant (PDBO-s: one dual per restart on the constraint
sum_i g(x_i) = 0, section 4 Discussion and the ablation table)."""
import numpy as np

import oracle as O
import workloads as W


def test_single_lagrangian_gradients_are_central_differences():
    """L_s is quadratic in x and linear in mu, so central differences are exact up to rounding."""
    Q, c = W.dense_qubo(12, seed=1)
    A, cp = O.canonicalize(Q, c)
    rng = np.random.default_rng(0)
    X = rng.random((3, 12))
    MU = np.array([2.5, -1.0, 0.0])
    L, GX, GMU = O.lagrangian_single(A, cp, X, MU)
    h = 1e-3
    for r in range(3):
        for k in (0, 5, 11):
            E = np.zeros_like(X)
            E[r, k] = h
            fd = (O.lagrangian_single(A, cp, X + E, MU)[0][r] - O.lagrangian_single(A, cp, X - E, MU)[0][r]) / (2 * h)
            assert abs(fd - GX[r, k]) <= 1e-7 * max(1.0, abs(GX[r, k]))
        dm = np.zeros(3)
        dm[r] = h
        fd = (O.lagrangian_single(A, cp, X, MU + dm)[0][r] - O.lagrangian_single(A, cp, X, MU - dm)[0][r]) / (2 * h)
        assert abs(fd - GMU[r]) <= 1e-9 * max(1.0, abs(GMU[r]))


def test_single_lagrangian_is_F_on_binary_points():
    """g vanishes at 0 and 1, so L_s(b, mu) = F(b) for every mu (as Prop. 3.1 for L)."""
    Q, c = W.dense_qubo(10, seed=2)
    A, cp = O.canonicalize(Q, c)
    rng = np.random.default_rng(1)
    Bits = rng.integers(0, 2, size=(6, 10))
    L, _, _ = O.lagrangian_single(A, cp, Bits.astype(np.float64), rng.normal(size=6) * 50)
    assert np.array_equal(L, O.objective_batch(Q, c, Bits).astype(np.float64))


def test_single_step_with_beta_zero_is_the_coordinate_step_with_equal_duals():
    """With beta = 0 the dual never moves, and mu in every coordinate is exactly the coordinate
    form with y_i = mu: same primal step, same perturbation rule."""
    Q, c = W.dense_qubo(30, seed=3)
    A, cp = O.canonicalize(Q, c)
    X, _ = O.init_state(30, 5, 7, 0.0)
    MU = np.array([3.0, 0.0, -2.0, -0.5, 10.0])
    for _ in range(40):
        Xs, MUs, Ds = O.gda_step_single(A, cp, X, MU, 0.02, 0.0, 0.05, 4.0)
        Xc, Yc, Dc = O.gda_step(A, cp, X, np.repeat(MU[:, None], 30, axis=1), 0.02, 0.0, 0.05, 4.0)
        assert np.array_equal(Xs, Xc) and np.array_equal(Ds, Dc)
        assert np.array_equal(MUs, MU) and np.array_equal(Yc, np.repeat(MU[:, None], 30, axis=1))
        X = Xs


def test_single_step_on_a_symmetric_instance_is_the_coordinate_step_with_beta_over_n():
    """Complete graph with equal weights, equal linear terms and equal starting coordinates: every
    coordinate of every iterate stays equal under both forms, the coordinate duals all equal y, and
    the single dual with step beta / n follows y (sum_i g(x_i) = n g(x)).  A wrong sign, a mean for
    the sum, or the new x in the dual step breaks this."""
    n = 16
    Q = 7 * (np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64))
    c = np.full(n, -100, dtype=np.int64)
    A, cp = O.canonicalize(Q, c)
    x0 = np.array([0.3, 0.5, 0.8, 0.1])
    X = np.repeat(x0[:, None], n, axis=1)
    Y = np.full((4, n), 40.0)
    MU = np.full(4, 40.0)
    beta, alpha = 2.0, 0.004
    for _ in range(300):
        Xc, Yc, _ = O.gda_step(A, cp, X, Y, alpha, beta, 0.01)
        Xs, MUs, _ = O.gda_step_single(A, cp, X, MU, alpha, beta / n, 0.01)
        assert np.allclose(Xs, Xc, rtol=0, atol=1e-12)
        assert np.allclose(MUs, Yc[:, 0], rtol=1e-12, atol=1e-12)
        assert np.all(Yc == Yc[:, :1])
        X, Y, MU = Xc, Yc, MUs
    assert np.all(MU < 40.0)           # the dual fell while x was fractional


def test_single_run_dual_is_monotone_and_bounded_per_step():
    """mu^{t+1} - mu^t = beta sum_i g(x_i^t) lies in [-n beta / 4, 0]; iterates stay in the box."""
    Q, c = W.dense_qubo(25, seed=4)
    p = W.dense_params(Q, restarts=6, iters=60, eval_every=10, seed=2)
    out = O.run(Q, c, p.restarts, 60, p.alpha, p.beta, p.ybar, p.delta, p.grad_tol, 10, p.seed,
                dump_iters=60, dual="single")
    mus = np.array(out["dumps"]["y"])
    xs = np.array(out["dumps"]["x"])
    assert mus.shape == (61, 6)
    dm = np.diff(mus, axis=0)
    assert np.all(dm <= 0.0) and np.all(dm >= -25 * p.beta / 4 - 1e-12)
    assert np.all((xs >= 0.0) & (xs <= 1.0))
    assert out["F_star"] == O.objective(Q, c, out["x_star"])
