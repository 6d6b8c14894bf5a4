"""Pins of the FP64 oracle against facts the paper and the mathematics fix (CPU only).

Each test names the passage it checks.  None of them re-derives a value with the oracle's own
formula: they use hand-worked fixtures (tests/golden), exhaustive enumeration, independent
definitions (edge counting, finite differences, KKT conditions) or the paper's invariants.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _bits(s):
    return np.array([int(ch) for ch in s], dtype=np.uint8)


# --------------------------------------------------------------------------------------
# objective, canonical form, multilinear extension
# --------------------------------------------------------------------------------------
def test_objective_and_canonical_form_match_hand_worked_fixture():
    g = _load("qubo_n3_hand.json")
    Q, c = np.array(g["Q"]), np.array(g["c"])
    for s, F in g["F_by_bits"].items():
        assert O.objective(Q, c, _bits(s)) == F
        assert O.objective_batch(Q, c, _bits(s)[None, :])[0] == F
    A, cp = O.canonicalize(Q, c)
    assert np.array_equal(A, np.array(g["A"], dtype=float))
    assert np.array_equal(cp, np.array(g["c_prime"], dtype=float))
    assert O.multilinear(A, cp, np.full(3, 0.5)) == g["f_at_half"]
    best, arg = O.brute_force(Q, c)
    assert best == g["min_F"]
    assert [O.bits_of(a, 3).tolist() for a in arg] == [_bits(g["argmin_bits"]).tolist()]


@pytest.mark.parametrize("n,seed", [(4, 1), (7, 2), (10, 3)])
def test_multilinear_closed_form_equals_bernoulli_expectation(n, seed):
    """Def. 2.2: f(x) = sum over xi of P_x(xi) F(xi); Prop. 2.4 gives the closed form."""
    rng = np.random.default_rng(seed)
    Q = rng.integers(-9, 10, size=(n, n))          # non-symmetric, non-zero diagonal
    c = rng.integers(-9, 10, size=n)
    A, cp = O.canonicalize(Q, c)
    for _ in range(3):
        x = rng.random(n)
        exp = 0.0
        for k in range(1 << n):
            xi = O.bits_of(k, n)
            p = np.prod(np.where(xi == 1, x, 1.0 - x))
            exp += p * O.objective(Q, c, xi)
        assert abs(O.multilinear(A, cp, x) - exp) <= 1e-9 * (1 + abs(exp))


def test_lemma_2_3_box_minimum_is_the_vertex_minimum():
    rng = np.random.default_rng(5)
    Q, c = W.dense_qubo(12, seed=3)
    A, cp = O.canonicalize(Q, c)
    best, _ = O.brute_force(Q, c)
    X = rng.random((4000, 12))
    f = 0.5 * np.einsum("ri,ri->r", X @ A, X) + X @ cp
    assert f.min() >= best - 1e-9


def test_maxcut_objective_is_minus_the_cut():
    """Section 4.1: cut(x) = sum_E w_ij (x_i + x_j - 2 x_i x_j); the QUBO has Q=W, c=-W1."""
    n = 30
    i, j, w = W.maxcut_er(n, mean_degree=5, seed=4)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    Qd = W.dense_from_csr(n, rowptr, col, val)
    rng = np.random.default_rng(0)
    for _ in range(20):
        b = rng.integers(0, 2, n).astype(np.uint8)
        cut = sum(int(ww) for a, bb, ww in zip(i, j, w) if b[a] != b[bb])
        assert O.objective(Qd, c, b) == -cut
        assert O.objective_csr(n, rowptr, col, val, c, b) == -cut


def test_mis_objective_counts_set_and_penalises_edges():
    """MIS appendix: maximise sum x_i - lambda sum_E x_i x_j (lambda = 4)."""
    n = 40
    rowptr, col, val, c, (i, j) = W.mis_regular(n, 3, seed=1)
    rng = np.random.default_rng(1)
    for _ in range(20):
        b = rng.integers(0, 2, n).astype(np.uint8)
        viol = int(np.sum(b[i] & b[j]))
        assert O.objective_csr(n, rowptr, col, val, c, b) == -int(b.sum()) + 4 * viol


# --------------------------------------------------------------------------------------
# Lagrangian and its gradients
# --------------------------------------------------------------------------------------
def test_lagrangian_equals_F_on_binary_points_for_any_dual():
    """Prop. 3.1 / g(0) = g(1) = 0: L(b, y) = F(b) whatever y is."""
    rng = np.random.default_rng(2)
    Q, c = W.dense_qubo(15, seed=9)
    A, cp = O.canonicalize(Q, c)
    Bm = rng.integers(0, 2, size=(16, 15)).astype(np.uint8)
    Y = rng.normal(scale=50.0, size=(16, 15))
    L, _, GY = O.lagrangian(A, cp, Bm.astype(float), Y)
    F = O.objective_batch(Q, c, Bm)
    assert np.array_equal(L, F.astype(float))
    assert np.all(GY == 0.0)


def test_gradients_match_central_finite_differences():
    """L is quadratic in x and linear in y, so central differences are exact up to rounding."""
    rng = np.random.default_rng(3)
    Q = rng.integers(-100, 101, size=(9, 9))
    c = rng.integers(-100, 101, size=9)
    A, cp = O.canonicalize(Q, c)
    X = rng.random((3, 9))
    Y = rng.normal(scale=10, size=(3, 9))
    _, GX, GY = O.lagrangian(A, cp, X, Y)
    h = 1e-3
    for r in range(3):
        for i in range(9):
            E = np.zeros_like(X)
            E[r, i] = h
            fx = (O.lagrangian(A, cp, X + E, Y)[0][r] - O.lagrangian(A, cp, X - E, Y)[0][r]) / (2 * h)
            fy = (O.lagrangian(A, cp, X, Y + E)[0][r] - O.lagrangian(A, cp, X, Y - E)[0][r]) / (2 * h)
            assert abs(fx - GX[r, i]) <= 1e-7 * (1 + abs(GX[r, i]))
            assert abs(fy - GY[r, i]) <= 1e-9


def test_maxcut_half_point_is_stationary_for_every_dual():
    """Example in section 3.2: x = 1/2 gives grad_x L = 0 exactly for Max-Cut, any y."""
    n = 50
    i, j, w = W.maxcut_er(n, 6, seed=7)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    A, cp = O.canonicalize(W.dense_from_csr(n, rowptr, col, val), c)
    Y = np.random.default_rng(0).normal(scale=5, size=(3, n))
    _, GX, _ = O.lagrangian(A, cp, np.full((3, n), 0.5), Y)
    assert np.all(GX == 0.0)


# --------------------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", range(3))
def test_gda_steps_match_hand_worked_iterations(case):
    g = _load("gda_steps_hand.json")["cases"][case]
    A, cp = O.canonicalize(np.array(g["Q"]), np.array(g["c"]))
    X = np.array(g["x0"])[None, :]
    Y = np.array(g["y0"])[None, :]
    for t in range(len(g["x"])):
        X, Y, D = O.gda_step(A, cp, X, Y, g["alpha"], g["beta"], g["delta"], g["grad_tol"])
        assert np.array_equal(D[0], np.array(g["d"][t])), (t, D)
        assert np.array_equal(X[0], np.array(g["x"][t])), (t, X)
        assert np.array_equal(Y[0], np.array(g["y"][t])), (t, Y)


def _run_small(T=600, n=24, B=8, seed=0):
    Q, c = W.dense_qubo(n, seed=seed)
    p = W.dense_params(Q, restarts=B, iters=T, eval_every=10, seed=seed)
    A, cp = O.canonicalize(Q, c)
    X, Y = O.init_state(n, B, p.seed, p.ybar)
    xs, ys = [X], [Y]
    for _ in range(T):
        X, Y, _ = O.gda_step(A, cp, X, Y, p.alpha, p.beta, p.delta, p.grad_tol)
        xs.append(X)
        ys.append(Y)
    return Q, c, A, cp, p, np.array(xs), np.array(ys)


def test_iterates_stay_in_box_and_duals_decrease_by_at_most_beta_over_4():
    """Eq. 5 projection keeps x in [0,1]^n; y^{t+1} - y^t = beta g(x^t) in [-beta/4, 0]."""
    _, _, _, _, p, xs, ys = _run_small()
    assert xs.min() >= 0.0 and xs.max() <= 1.0
    dy = np.diff(ys, axis=0)
    assert dy.max() <= 0.0
    assert dy.min() >= -p.beta / 4 * (1 + 1e-12)


def test_dual_telescoping_identity():
    """Proof of Thm. 3.7: y^T = y^0 + beta * sum_{t<T} g(x^t)."""
    _, _, _, _, p, xs, ys = _run_small(T=300)
    lhs = ys[-1]
    rhs = ys[0] + p.beta * np.sum(xs[:-1] ** 2 - xs[:-1], axis=0)
    assert np.max(np.abs(lhs - rhs)) <= 1e-9 * np.max(np.abs(ys[0]))


def test_dual_lower_bound_of_prop_3_3():
    """Prop. 3.3 with Theta bounded by sum_i (sum_j |A_ij| + |c'_i|) >= max ||grad f||_1."""
    n, B, T = 16, 8, 4000
    Q, c = W.dense_qubo(n, seed=1, lo=-3, hi=3)
    A, cp = O.canonicalize(Q, c)
    alpha, beta, delta, ybar = 0.05, 0.05, 0.05, 2.0
    X, Y = O.init_state(n, B, 11, ybar)
    theta = float(np.sum(np.abs(A)) + np.sum(np.abs(cp)))
    bound = (1 + theta) / (2 * (0.5 - delta) - 1) + (2 + math.ceil(1 / (2 * alpha))) * beta * (-0.25)
    ymin = np.inf
    for _ in range(T):
        X, Y, _ = O.gda_step(A, cp, X, Y, alpha, beta, delta, 2 * delta)
        ymin = min(ymin, Y.min())
    assert ymin >= bound


def test_iterates_converge_to_binary_points():
    """Cor. 3.5 / Def. 3.6: long runs reach epsilon-binary points."""
    n, B = 20, 8
    Q, c = W.dense_qubo(n, seed=2)
    p = W.dense_params(Q, restarts=B, iters=4000, seed=2)
    A, cp = O.canonicalize(Q, c)
    X, Y = O.init_state(n, B, p.seed, p.ybar)
    for _ in range(p.iters):
        X, Y, _ = O.gda_step(A, cp, X, Y, p.alpha, p.beta, p.delta, p.grad_tol)
    frac = -np.sum(X * X - X, axis=1)           # -sum g(x_i), Def. 3.6
    assert np.all(frac <= 1e-4)
    assert np.all((X < 1e-4) | (X > 1 - 1e-4))


def test_convex_case_converges_to_the_box_qp_minimiser():
    """Section 4.4: with beta = 0 and A + 2 ybar I positive definite, GDA is projected gradient
    on a strictly convex quadratic; its limit satisfies the KKT conditions of the box QP."""
    n, B = 12, 4
    Q, c = W.dense_qubo(n, seed=4, lo=-5, hi=5)
    A, cp = O.canonicalize(Q, c)
    lam = np.linalg.eigvalsh(A)
    ybar = -lam.min() / 2 + 1.0
    H = A + 2 * ybar * np.eye(n)
    alpha = 1.0 / np.linalg.eigvalsh(H).max()
    X, Y = O.init_state(n, B, 3, ybar)
    for _ in range(20000):
        X, Y, _ = O.gda_step(A, cp, X, Y, alpha, 0.0, 0.01, 0.02)
    assert np.max(np.abs(X - X[0])) <= 1e-9            # unique minimiser
    x = X[0]
    grad = H @ x + cp - ybar                            # d/dx of f(x) + ybar * sum(x^2 - x)
    free = (x > 1e-9) & (x < 1 - 1e-9)
    assert np.all(np.abs(grad[free]) <= 1e-7)
    assert np.all(grad[x <= 1e-9] >= -1e-7)
    assert np.all(grad[x >= 1 - 1e-9] <= 1e-7)


def test_scale_invariance_is_bitwise_for_powers_of_two():
    """(A, c', ybar, alpha, beta, tol) -> (sA, sc', s ybar, alpha/s, s beta, s tol) leaves x fixed."""
    Q, c = W.dense_qubo(16, seed=6)
    A, cp = O.canonicalize(Q, c)
    X, Y = O.init_state(16, 4, 1, 300.0)
    X2, Y2 = X.copy(), Y * 8
    for _ in range(200):
        X, Y, _ = O.gda_step(A, cp, X, Y, 1e-4, 5.0, 0.01, 2.0)
        X2, Y2, _ = O.gda_step(8 * A, 8 * cp, X2, Y2, 1e-4 / 8, 40.0, 0.01, 16.0)
    assert np.array_equal(X, X2)
    assert np.array_equal(Y * 8, Y2)


# --------------------------------------------------------------------------------------
# x^0 generator, rounding, best tracking
# --------------------------------------------------------------------------------------
def test_splitmix64_matches_published_outputs():
    g = _load("splitmix64_vectors.json")
    for seed, outs in g["outputs"].items():
        got = O.splitmix64_stream(int(seed), np.arange(len(outs)))
        assert [int(v) for v in got] == [int(v, 0) for v in outs]


def test_uniform_start_is_24_bit_and_uniform():
    X, Y = O.init_state(1000, 16, 42, 6.0)
    assert np.all((X >= 0) & (X < 1))
    assert np.array_equal(X * 2**24, np.floor(X * 2**24))
    assert np.all(X.astype(np.float32).astype(np.float64) == X)
    assert abs(X.mean() - 0.5) < 0.01 and abs(X.var() - 1 / 12) < 0.01
    assert np.all(Y == 6.0)
    assert not np.array_equal(X[0], X[1])


def test_run_finds_the_brute_force_optimum_and_reports_a_true_candidate():
    n = 16
    Q, c = W.dense_qubo(n, seed=8)
    p = W.dense_params(Q, restarts=32, iters=1000, eval_every=10, seed=0)
    out = O.run(Q, c, **p.asdict())
    best, arg = O.brute_force(Q, c)
    assert out["F_star"] >= best
    assert O.objective(Q, c, out["x_star"]) == out["F_star"]
    # every per-restart best is an actual evaluation with that F
    for r in range(p.restarts):
        t = out["best_t"][r]
        Fs = dict(out["evals"])[t]
        assert Fs[r] == out["best_F"][r]
    assert out["F_star"] == best          # 32 restarts reach the optimum of this instance


def test_best_tracking_tie_rules_by_brute_force():
    """Global best = lexicographic min of (F, t, r) over all evaluations; per restart, ties keep
    the earliest t (strict improvement only)."""
    n = 10
    Q, c = W.dense_qubo(n, seed=12, lo=-2, hi=2)         # small alphabet: many ties
    p = W.dense_params(Q, restarts=12, iters=300, eval_every=7, seed=3)
    out = O.run(Q, c, **p.asdict())
    allv = [(int(F[r]), t, r) for t, F in out["evals"] for r in range(p.restarts)]
    Fm, tm, rm = min(allv)
    assert (out["F_star"], out["t_star"], out["r_star"]) == (Fm, tm, rm)
    for r in range(p.restarts):
        Fr = min(v for v in allv if v[2] == r)
        assert (out["best_F"][r], out["best_t"][r]) == (Fr[0], Fr[1])
    assert [t for t, _ in out["evals"]] == list(range(7, 300, 7)) + [300]


@pytest.mark.parametrize("n,d", [(400, 3), (500, 100)])
def test_regular_graph_generator_is_simple_and_regular(n, d):
    """The MIS and Max-Cut stand-ins need simple d-regular graphs (pairing model; edge switches
    for large d)."""
    rowptr, col, val, c, (i, j) = W.mis_regular(n, d, seed=5)
    assert np.all(np.diff(rowptr) == d)
    assert np.all(i != j)
    key = np.minimum(i, j).astype(np.int64) * n + np.maximum(i, j)
    assert np.unique(key).size == key.size == n * d // 2


def test_csr_canonical_form_equals_the_dense_one():
    """canonicalize_csr (scipy storage) gives the same A, c' as canonicalize on the dense Q."""
    n = 60
    rng = np.random.default_rng(4)
    Qd = rng.integers(-5, 6, size=(n, n)) * (rng.random((n, n)) < 0.2)   # non-symmetric, diagonal
    c = rng.integers(-5, 6, size=n)
    rows, cols = np.nonzero(Qd)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    A_s, cp_s = O.canonicalize_csr(n, rowptr, cols, Qd[rows, cols], c)
    A_d, cp_d = O.canonicalize(Qd, c)
    assert np.array_equal(A_s.toarray(), A_d) and np.array_equal(cp_s, cp_d)
    X = rng.random((3, n))
    Y = rng.normal(size=(3, n))
    for a, b in zip(O.lagrangian(A_s, cp_s, X, Y), O.lagrangian(A_d, cp_d, X, Y)):
        assert np.allclose(a, b, rtol=1e-13, atol=1e-12)
