"""Randomised pins of the oracle (hypothesis): properties the paper's statements fix on every small
instance, checked against exhaustive enumeration rather than against the oracle's own formulas.

* Prop. 2.4: the canonical multilinear form equals F at every binary point.
* Def. 2.2: the multilinear extension is the expectation of F under independent Bernoulli(x_i).
* Prop. 3.1: at binary points the Lagrangian equals F, whatever the duals.
* Algorithm 1: an iteration keeps x in the box, and with g <= 0 on the box the dual never rises.
* The dual certificate: with L(., ybar) convex on the box, the bound it returns from any box point
  lies below the brute-force minimum of F.
* The sparse objective of a CSR matrix equals the dense objective of the same matrix.
"""
import itertools

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle.pdbo as O  # noqa: E402

SETTINGS = settings(max_examples=60, deadline=None)


@st.composite
def qubo(draw, n_max=7, lo=-9, hi=9):
    n = draw(st.integers(1, n_max))
    seed = draw(st.integers(0, 2**32 - 1))
    rng = np.random.default_rng(seed)
    Q = rng.integers(lo, hi + 1, size=(n, n)).astype(np.int64)
    c = rng.integers(3 * lo, 3 * hi + 1, size=n).astype(np.int64)
    return Q, c, rng


def all_bits(n):
    return np.array(list(itertools.product((0, 1), repeat=n)), dtype=np.int64)


@SETTINGS
@given(qubo())
def test_canonical_form_equals_F_on_every_binary_point(case):
    Q, c, _ = case
    A, cp = O.canonicalize(Q, c)
    for b in all_bits(Q.shape[0]):
        assert O.multilinear(A, cp, b) == pytest.approx(float(b @ Q @ b + c @ b), abs=1e-9)


@SETTINGS
@given(qubo(n_max=6))
def test_multilinear_extension_is_the_bernoulli_expectation(case):
    Q, c, rng = case
    n = Q.shape[0]
    A, cp = O.canonicalize(Q, c)
    x = rng.uniform(0.0, 1.0, size=n)
    expect = 0.0
    for b in all_bits(n):
        p = np.prod(np.where(b == 1, x, 1.0 - x))
        expect += p * float(b @ Q @ b + c @ b)
    assert O.multilinear(A, cp, x) == pytest.approx(expect, rel=1e-9, abs=1e-9)


@SETTINGS
@given(qubo())
def test_lagrangian_equals_F_at_binary_points_for_any_dual(case):
    Q, c, rng = case
    n = Q.shape[0]
    A, cp = O.canonicalize(Q, c)
    Bm = all_bits(n)
    Y = rng.normal(scale=50.0, size=Bm.shape)
    L, _, GY = O.lagrangian(A, cp, Bm.astype(np.float64), Y)
    F = np.einsum("ri,ri->r", Bm @ Q.T, Bm) + Bm @ c
    assert np.allclose(L, F, rtol=0, atol=1e-9)
    assert np.all(GY == 0.0)   # g vanishes exactly at 0 and 1


@SETTINGS
@given(qubo(), st.floats(1e-4, 0.5), st.floats(0.0, 2.0), st.floats(0.0, 0.2))
def test_an_iteration_keeps_x_in_the_box_and_never_raises_the_dual(case, alpha, beta, delta):
    Q, c, rng = case
    n = Q.shape[0]
    A, cp = O.canonicalize(Q, c)
    X = rng.uniform(0.0, 1.0, size=(5, n))
    Y = rng.normal(scale=10.0, size=(5, n))
    Xn, Yn, _ = O.gda_step(A, cp, X, Y, alpha, beta, delta)
    assert np.all((Xn >= 0.0) & (Xn <= 1.0))
    assert np.all(Yn <= Y + 1e-15)   # y <- y + beta (x^2 - x) with x in [0, 1]


@SETTINGS
@given(qubo(n_max=8), st.floats(0.0, 5.0))
def test_certificate_never_exceeds_the_minimum(case, extra):
    Q, c, rng = case
    n = Q.shape[0]
    A, cp = O.canonicalize(Q, c)
    # L(., ybar) = 1/2 x^T (A + 2 ybar I) x + (c' - ybar 1)^T x is convex once 2 ybar >= -lambda_min(A)
    ybar = max(0.0, -np.linalg.eigvalsh(A)[0] / 2.0) + extra
    F_min, _ = O.brute_force(Q, c)
    for _ in range(4):
        x = rng.uniform(0.0, 1.0, size=n)
        assert O.certificate(A, cp, ybar, x) <= F_min + 1e-7 * max(1.0, abs(F_min))


@SETTINGS
@given(qubo(n_max=9), st.floats(0.05, 0.9))
def test_sparse_objective_matches_the_dense_one(case, density):
    Q, c, rng = case
    n = Q.shape[0]
    Qs = np.where(rng.uniform(size=Q.shape) < density, Q, 0)
    rows, cols = np.nonzero(Qs)
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
    order = np.lexsort((cols, rows))
    col, val = cols[order], Qs[rows[order], cols[order]]
    for b in all_bits(min(n, 9))[:64]:
        bb = np.zeros(n, np.int64)
        bb[:len(b)] = b
        assert O.objective_csr(n, rowptr, col, val, c, bb) == O.objective(Qs, c, bb)
