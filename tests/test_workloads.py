"""The seeded input generators produce the workloads their recipes describe (shapes, value ranges,
structure) and the same instance for the same seed; they hold none of the method's arithmetic."""
import numpy as np
import pytest

import workloads as W


def test_dense_qubo_recipe_and_reproducibility():
    Q, c = W.dense_qubo(300, seed=7)
    Q2, c2 = W.dense_qubo(300, seed=7)
    assert np.array_equal(Q, Q2) and np.array_equal(c, c2)
    assert Q.dtype == np.int32 and c.dtype == np.int32 and Q.shape == (300, 300)
    assert np.array_equal(Q, Q.T) and np.all(np.diagonal(Q) == 0)
    assert Q.min() >= -100 and Q.max() <= 100 and c.min() >= -100 and c.max() <= 100
    off = Q[np.triu_indices(300, 1)]
    assert abs(off.mean()) < 2.0 and 50 < off.std() < 65           # uniform on [-100, 100]: std 58
    assert not np.array_equal(W.dense_qubo(300, seed=8)[0], Q)


@pytest.mark.parametrize("density", [0.05, 0.5])
def test_dense_qubo_density_mask(density):
    Q, _ = W.dense_qubo(400, seed=1, density=density)
    off = Q[np.triu_indices(400, 1)]
    frac = np.mean(off != 0)
    assert abs(frac - density * (200 / 201)) < 0.02                  # zero entries of U{-100..100}
    assert np.array_equal(Q, Q.T)


def test_erdos_renyi_mean_degree_and_weights():
    n = 4000
    i, j, w = W.maxcut_er(n, 6.0, seed=0)
    assert np.all(i < j) and len(set(zip(i.tolist(), j.tolist()))) == i.size     # simple graph
    assert abs(2 * i.size / n - 6.0) < 0.2
    assert set(np.unique(w).tolist()) <= {-1, 1}
    i2, j2, w2 = W.maxcut_er(n, 6.0, seed=0)
    assert np.array_equal(i, i2) and np.array_equal(j, j2) and np.array_equal(w, w2)


def test_torus_is_four_regular_with_periodic_neighbours():
    rows, cols = 7, 9
    i, j, w = W.maxcut_torus(rows, cols, seed=2)
    n = rows * cols
    assert i.size == 2 * n
    deg = np.bincount(np.concatenate([i, j]), minlength=n)
    assert np.all(deg == 4)
    pairs = {(int(a), int(b)) for a, b in zip(i, j)}
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            right, down = r * cols + (c + 1) % cols, ((r + 1) % rows) * cols + c
            assert (min(v, right), max(v, right)) in pairs and (min(v, down), max(v, down)) in pairs


def test_maxcut_qubo_is_the_weight_matrix_and_minus_its_row_sums():
    n = 50
    i, j, w = W.maxcut_er(n, 6.0, seed=3)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    Q = W.dense_from_csr(n, rowptr, col, val)
    Wm = np.zeros((n, n), np.int64)
    Wm[i, j] = w
    Wm[j, i] = w
    assert np.array_equal(Q, Wm)
    assert np.array_equal(c, -Wm.sum(axis=1))
    assert np.all(np.diff(rowptr) >= 0) and rowptr[-1] == col.size
    for r in range(n):
        cols = col[rowptr[r]:rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)                                # sorted, no duplicates


def test_mis_instance_penalises_each_edge_by_lambda():
    n, d, lam = 60, 3, 4
    rowptr, col, val, c, (i, j) = W.mis_regular(n, d, seed=0, lam=lam)
    Q = W.dense_from_csr(n, rowptr, col, val)
    assert np.all(c == -1)
    assert np.all(np.bincount(np.concatenate([i, j]), minlength=n) == d)
    # x^T Q x counts lam per edge with both ends chosen
    x = np.zeros(n, np.int64)
    x[[i[0], j[0]]] = 1
    assert int(x @ Q @ x) == lam
