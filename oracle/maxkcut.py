"""FP64 CPU oracle of PDBO's generalisation to Max-k-Cut (appendix on Max-k-Cut).

TEST INFRASTRUCTURE ONLY, like ``oracle.pdbo``: only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU leg of ``bench.py`` may import it; it shares no code with the CUDA path.

Each vertex i carries a point X_:,i of the probability simplex written as softmax(Z_:,i).  With
the symmetric weight matrix W and the quadratic constraint function g(X_:,i) = sum_j X_ji^2 - 1
(zero exactly at the vertices e^(j) of the simplex, negative elsewhere on it) the Lagrangian is

    L(X, y) = Tr(X W X^T) + sum_i y_i g(X_:,i),

and the method runs the simultaneous gradient descent-ascent of section 3.2 on (Z, y):

    Z <- Z - alpha dL/dZ (Z, y),        y <- y + beta g(X)          (both at the old point).

Batched arrays are restart-major: ``Z[r, i, j]`` is logit j of vertex i in restart r.  W is a
scipy sparse or dense symmetric float matrix without diagonal.

==================  ===============================================  ===========================
function            follows                                          pinned by
==================  ===============================================  ===========================
softmax             the reparametrisation of the appendix            rows on the simplex; shift
                                                                     invariance
lagrangian_k        L above                                          k = 2 equals twice the
                                                                     Max-Cut Lagrangian plus a
                                                                     constant; L = Tr(XWX^T) =
                                                                     2 W_E - 2 cut on vertices
grad_z              chain rule through the softmax                   central finite differences
gda_step_k          simultaneous GDA (Eq. 5) on (Z, y)               dual monotone (g <= 0);
                                                                     X stays on the simplex
round_parts / cut   argmax part (ties to the smallest index), cut =  direct edge enumeration;
                    sum of w over edges across parts                 brute force over k^n
run_k               best-of-B retention (section 4.2)                finds the optimum of small
                                                                     graphs (brute force)
==================  ===============================================  ===========================
"""
from __future__ import annotations

import itertools

import numpy as np

from .pdbo import uniform24


def softmax(Z):
    """X_:,i = softmax(Z_:,i) along the last axis (shifted by the maximum; the value is the same)."""
    Z = np.asarray(Z, dtype=np.float64)
    E = np.exp(Z - Z.max(axis=-1, keepdims=True))
    return E / E.sum(axis=-1, keepdims=True)


def _wx(W, X):
    """(W X_r)_i,j = sum_l W_il X_r,l,j for every restart (X: B x n x k)."""
    B, n, k = X.shape
    M = np.asarray(W @ X.transpose(1, 0, 2).reshape(n, B * k))
    return M.reshape(n, B, k).transpose(1, 0, 2)


def lagrangian_k(W, X, Y):
    """Value and gradients of L(X, y) = Tr(X W X^T) + sum_i y_i (|X_:,i|^2 - 1).

    Returns ``(L[B], dL/dX [B, n, k], dL/dy [B, n])`` with dL/dX_:,i = 2 (W X)_i + 2 y_i X_:,i
    (W symmetric) and dL/dy_i = |X_:,i|^2 - 1."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    WX = _wx(W, X)
    G = np.sum(X * X, axis=2) - 1.0
    Lval = np.einsum("rij,rij->r", X, WX) + np.sum(Y * G, axis=1)
    GX = 2.0 * WX + 2.0 * Y[:, :, None] * X
    return Lval, GX, G


def grad_z(W, Z, Y):
    """dL/dZ through the softmax: for s = X_:,i and h = dL/dX_:,i, dL/dZ_:,i = s * (h - <s, h>)."""
    X = softmax(Z)
    _, GX, G = lagrangian_k(W, X, Y)
    dot = np.sum(X * GX, axis=2, keepdims=True)
    return X * (GX - dot), X, G


def init_state_k(n, k, B, seed, ybar):
    """Z^0_{r,i,j} = U(seed, r, i k + j) (the generator of x^0, one draw per logit); y^0 = ybar."""
    r = np.arange(B, dtype=np.uint64)[:, None]
    q = np.arange(n * k, dtype=np.uint64)[None, :]
    Z = uniform24(seed, r, q).reshape(B, n, k)
    return Z, np.full((B, n), float(ybar))


def gda_step_k(W, Z, Y, alpha, beta):
    """One simultaneous GDA step on (Z, y).  Returns (Z^{t+1}, Y^{t+1}, dL/dZ at t)."""
    DZ, X, G = grad_z(W, Z, Y)
    return np.asarray(Z, dtype=np.float64) - alpha * DZ, np.asarray(Y, dtype=np.float64) + beta * G, DZ


def round_parts(X):
    """Part of every vertex: argmax_j X_:,i, ties to the smallest j."""
    return np.argmax(np.asarray(X), axis=-1).astype(np.uint8)


def cut_value(i, j, w, parts):
    """sum of w_e over the edges e = (i, j) (each listed once) whose ends lie in different parts;
    one value for parts of shape (n,), one per row for shape (B, n)."""
    parts = np.asarray(parts)
    w = np.asarray(w, dtype=np.int64)
    if parts.ndim == 1:
        return int(np.sum(w * (parts[i] != parts[j])))
    return np.sum(w[None, :] * (parts[:, i] != parts[:, j]), axis=1)


def weight_matrix(n, i, j, w):
    """Symmetric W (scipy CSR, float64) of an edge list given once per edge."""
    import scipy.sparse as sp
    M = sp.coo_matrix((np.asarray(w, dtype=np.float64), (np.asarray(i), np.asarray(j))), shape=(n, n))
    return (M + M.T).tocsr()


def brute_force_k(n, k, i, j, w):
    """Maximum cut over all k^n assignments (n small) and one maximiser."""
    best, arg = None, None
    for p in itertools.product(range(k), repeat=n):
        v = cut_value(i, j, w, np.array(p))
        if best is None or v > best:
            best, arg = v, np.array(p, dtype=np.uint8)
    return best, arg


def run_k(n, k, i, j, w, restarts, iters, alpha, beta, ybar, eval_every=10, seed=0, Z0=None):
    """Batched PDBO for Max-k-Cut: B restarts, candidates round_parts(softmax(Z^t)) evaluated at
    t = K, 2K, ... and T; per restart the best cut is kept with its earliest t (strict
    improvement); F = -cut, and the global best is the lexicographic minimum of (F, t, r)."""
    from .pdbo import eval_points
    W = weight_matrix(n, i, j, w)
    Z, Y = init_state_k(n, k, restarts, seed, ybar)
    if Z0 is not None:
        Z = np.array(Z0, dtype=np.float64)
    pts = set(eval_points(iters, eval_every))
    best_F = np.full(restarts, np.iinfo(np.int64).max, dtype=np.int64)
    best_t = np.full(restarts, -1, dtype=np.int64)
    best_parts = np.zeros((restarts, n), dtype=np.uint8)
    for t in range(iters):
        Z, Y, _ = gda_step_k(W, Z, Y, alpha, beta)
        if t + 1 in pts:
            parts = round_parts(softmax(Z))
            F = -cut_value(i, j, w, parts)
            better = F < best_F
            best_F[better] = F[better]
            best_t[better] = t + 1
            best_parts[better] = parts[better]
    order = np.lexsort((np.arange(restarts), best_t, best_F))
    r = int(order[0])
    return {"Z": Z, "Y": Y, "best_F": best_F, "best_t": best_t, "best_parts": best_parts,
            "F_star": int(best_F[r]), "t_star": int(best_t[r]), "r_star": r, "parts_star": best_parts[r].copy()}
