"""Pins of the Max-k-Cut oracle (appendix on Max-k-Cut: softmax reparametrisation of the simplex,
quadratic constraint function, simultaneous GDA)."""
import numpy as np

import oracle as O
import oracle.maxkcut as K
import workloads as W


def _graph(n, m, seed, weights="pm1"):
    rng = np.random.default_rng(seed)
    pairs = set()
    while len(pairs) < m:
        a, b = sorted(rng.choice(n, size=2, replace=False))
        pairs.add((int(a), int(b)))
    i, j = (np.array(v, dtype=np.int32) for v in zip(*sorted(pairs)))
    w = rng.choice([-1, 1], size=m).astype(np.int32) if weights == "pm1" else np.ones(m, np.int32)
    return i, j, w


def test_softmax_rows_lie_on_the_simplex_and_ignore_shifts():
    rng = np.random.default_rng(0)
    Z = rng.normal(scale=3.0, size=(4, 9, 5))
    X = K.softmax(Z)
    assert np.all(X > 0) and np.allclose(X.sum(axis=2), 1.0, atol=1e-15)
    assert np.allclose(K.softmax(Z + 17.0), X, atol=1e-15)


def test_two_parts_is_twice_the_max_cut_lagrangian_plus_the_total_weight():
    """k = 2 with X_:,i = (x_i, 1 - x_i): Tr(X W X^T) = 2 f(x) + 1^T W 1 with f the Max-Cut
    multilinear form, and g_quad(X_:,i) = 2 g(x_i); so L_2 = 2 L + 1^T W 1 against the pinned
    Max-Cut oracle."""
    n = 40
    i, j, w = _graph(n, 90, seed=1)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    A, cp = O.canonicalize_csr(n, rowptr, col, val, c)
    Wm = K.weight_matrix(n, i, j, w)
    rng = np.random.default_rng(2)
    x = rng.uniform(0.05, 0.95, size=(3, n))
    y = rng.normal(scale=4.0, size=(3, n))
    X2 = np.stack([x, 1.0 - x], axis=2)
    Lk, GXk, Gk = K.lagrangian_k(Wm, X2, y)
    L1, GX1, G1 = O.lagrangian(A, cp, x, y)
    assert np.allclose(Lk, 2.0 * L1 + Wm.sum(), rtol=0, atol=1e-9)
    assert np.allclose(Gk, 2.0 * G1, atol=1e-15)
    # the derivative along x of L_2 is dL/dX_0 - dL/dX_1, which must equal 2 dL/dx
    assert np.allclose(GXk[:, :, 0] - GXk[:, :, 1], 2.0 * GX1, atol=1e-9)


def test_lagrangian_on_vertices_is_the_trace_form_of_the_cut():
    """On one-hot X every g vanishes and Tr(X W X^T) = 1^T W 1 - 2 cut, for any y."""
    n, k = 30, 4
    i, j, w = _graph(n, 70, seed=3)
    Wm = K.weight_matrix(n, i, j, w)
    rng = np.random.default_rng(4)
    parts = rng.integers(0, k, size=(5, n))
    X = np.eye(k)[parts]
    L, _, G = K.lagrangian_k(Wm, X, rng.normal(scale=9.0, size=(5, n)))
    assert np.all(G == 0.0)
    cut = K.cut_value(i, j, w, parts)
    assert np.array_equal(L, Wm.sum() - 2.0 * cut)
    # the cut itself by direct enumeration of the edges
    for r in range(5):
        assert cut[r] == sum(int(ww) for a, b, ww in zip(i, j, w) if parts[r, a] != parts[r, b])


def test_grad_z_is_the_central_difference_of_the_lagrangian():
    n, k = 12, 3
    i, j, w = _graph(n, 25, seed=5)
    Wm = K.weight_matrix(n, i, j, w)
    rng = np.random.default_rng(6)
    Z = rng.normal(size=(2, n, k))
    Y = rng.normal(scale=3.0, size=(2, n))
    DZ, _, _ = K.grad_z(Wm, Z, Y)
    h = 1e-6
    for r, a, b in ((0, 0, 0), (1, 5, 2), (0, 11, 1), (1, 3, 0)):
        E = np.zeros_like(Z)
        E[r, a, b] = h
        Lp = K.lagrangian_k(Wm, K.softmax(Z + E), Y)[0][r]
        Lm = K.lagrangian_k(Wm, K.softmax(Z - E), Y)[0][r]
        assert abs((Lp - Lm) / (2 * h) - DZ[r, a, b]) <= 1e-6 * max(1.0, abs(DZ[r, a, b]))


def test_gda_keeps_the_simplex_and_a_falling_dual():
    """g <= 0 on the simplex (sum X^2 >= 1/k), so y^{t+1} - y^t lies in [beta (1/k - 1), 0]."""
    n, k = 50, 3
    i, j, w = _graph(n, 120, seed=7)
    Wm = K.weight_matrix(n, i, j, w)
    Z, Y = K.init_state_k(n, k, 6, 3, 6.0)
    beta = 0.05
    for _ in range(200):
        Zn, Yn, _ = K.gda_step_k(Wm, Z, Y, 0.05, beta)
        dY = Yn - Y
        assert np.all(dY <= 0.0) and np.all(dY >= beta * (1.0 / k - 1.0) - 1e-15)
        Z, Y = Zn, Yn
    X = K.softmax(Z)
    assert np.allclose(X.sum(axis=2), 1.0, atol=1e-12)


def test_initial_logits_are_the_counter_based_uniform_draws():
    Z, Y = K.init_state_k(5, 3, 2, 11, 6.0)
    X0, _ = O.init_state(15, 2, 11, 0.0)      # the same stream, index i k + j
    assert np.array_equal(Z.reshape(2, 15), X0) and np.all(Y == 6.0)


def test_run_finds_the_brute_force_max_k_cut_of_small_graphs():
    for seed, (n, m, k) in enumerate(((8, 14, 3), (7, 12, 3), (9, 16, 4))):
        i, j, w = _graph(n, m, seed=10 + seed, weights="unit")
        best, _ = K.brute_force_k(n, k, i, j, w)
        out = K.run_k(n, k, i, j, w, restarts=48, iters=1500, alpha=0.01, beta=0.01, ybar=6.0,
                      eval_every=10, seed=seed)
        assert out["F_star"] == -best
        assert K.cut_value(i, j, w, out["parts_star"]) == best


def test_hand_worked_step_takes_both_updates_at_the_old_point():
    """One step worked by hand (k = 3, two vertices joined by one edge of weight 1; the updates of
    section 3.2 / Eq. 5, simultaneous):

    Z_:,0 = (0, ln 2, ln 5)  ->  s0 = softmax = (1, 2, 5)/8;   y0 = 1
    Z_:,1 = (ln 3, 0, ln 4)  ->  s1 = (3, 1, 4)/8;             y1 = 2
    dL/dX_:,i = 2 (W X)_i + 2 y_i s_i:   h0 = 2 s1 + 2 s0 = (1, 3/4, 9/4),
                                         h1 = 2 s0 + 4 s1 = (7/4, 1, 13/4)
    dL/dZ_:,i = s_i * (h_i - <s_i, h_i>):  <s0, h0> = 55/32, <s1, h1> = 77/32
        dZ0 = (-23/256, -31/128, 85/256),   dZ1 = (-63/256, -45/256, 27/64)
    g_i = |s_i|^2 - 1:  g0 = 30/64 - 1 = -17/32,  g1 = 26/64 - 1 = -19/32
    alpha = 1/2, beta = 1/4:  Z' - Z = -alpha dZ,  y' = y + beta g(s) at the OLD point:
        y0' = 1 - 17/128 = 111/128,  y1' = 2 - 19/128 = 237/128.
    Taking the dual step at the new point softmax(Z') instead changes y' by about 1e-2."""
    Wm = K.weight_matrix(2, np.array([0]), np.array([1]), np.array([1]))
    Z = np.array([[[0.0, np.log(2.0), np.log(5.0)], [np.log(3.0), 0.0, np.log(4.0)]]])
    Y = np.array([[1.0, 2.0]])
    Zn, Yn, DZ = K.gda_step_k(Wm, Z, Y, 0.5, 0.25)
    dz = np.array([[[-23 / 256, -31 / 128, 85 / 256], [-63 / 256, -45 / 256, 27 / 64]]])
    assert np.max(np.abs(DZ - dz)) <= 1e-12
    assert np.max(np.abs((Zn - Z) + 0.5 * dz)) <= 1e-12
    assert np.max(np.abs(Yn - np.array([[111 / 128, 237 / 128]]))) <= 1e-12
    # the same step at the new point would be visibly different: the pin can tell them apart
    Gnew = np.sum(K.softmax(Zn) ** 2, axis=2) - 1.0
    assert np.min(np.abs((Y + 0.25 * Gnew) - Yn)) > 1e-3
