"""Seeded instance generators (no PDBO arithmetic lives here).

Every generator takes an integer ``seed`` and draws from numpy's PCG64 keyed by
``(seed, tag)``, where the tag separates the kinds of instance, so the same seed gives the
same instance on every machine.

Instance recipes (the paper's Gset and CNF sets are not available, so these synthetic
families stand in for its workloads, with the same sizes and weight alphabets):

* dense QUBO: a symmetric integer matrix M with entries uniform in [lo, hi]; the diagonal
  becomes the linear term (``c = diag M``) and ``Q = M - diag(M)``, so that
  ``F(x) = x^T Q x + c^T x`` equals ``x^T M x`` on binary points.  Optional density masks
  off-diagonal pairs symmetrically.
* Max-Cut: an undirected weighted graph W (Erdos-Renyi, 2-D torus, or random d-regular
  from the pairing model) written as the QUBO ``Q = W`` (stored in both directions) and
  ``c = -W 1``, so that ``F(x) = -cut(x)`` (paper section 4.1 and the minimisation form in
  section 4.4).
* MIS: ``F(x) = -sum x_i + lambda * sum_{(i,j) in E} x_i x_j`` with lambda = 4 (paper,
  appendix on MIS), i.e. ``Q_ij = Q_ji = lambda/2`` on edges and ``c = -1``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_TAG_DENSE = 11
_TAG_ER = 12
_TAG_TORUS = 13
_TAG_REGULAR = 14
_TAG_HETERO = 15
_TAG_MIS = 16


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & (2**63 - 1), tag]))


# ----------------------------------------------------------------------------------------
# dense QUBO
# ----------------------------------------------------------------------------------------
def dense_qubo(n: int, seed: int = 0, lo: int = -100, hi: int = 100, density: float = 1.0,
               rng: np.random.Generator | None = None, dtype=np.int32):
    """Return ``(Q, c)``: ``Q`` n x n symmetric with zero diagonal (``dtype``: int32, or int8 for
    the entries drawn here, which all fit), ``c`` int32 n.

    ``M`` is symmetric with every upper-triangle entry (diagonal included) uniform in
    ``[lo, hi]``; pairs ``i < j`` are kept with probability ``density``; ``c = diag(M)``.
    The draws: an n x n int8 matrix R (row-major), then, if density < 1, a uint32 per entry in
    blocks of 2048 rows (kept when below density * 2^32); M takes R's upper triangle.
    """
    if not (-128 <= lo <= hi <= 127):
        raise ValueError("dense_qubo draws int8 entries; use lo, hi within [-128, 127]")
    if rng is None:
        rng = _rng(seed, _TAG_DENSE)
    R = rng.integers(lo, hi + 1, size=(n, n), dtype=np.int8)
    if density < 1.0:
        blk = 2048
        thr = np.uint32(min(int(density * 2**32), 2**32 - 1))
        for r0 in range(0, n, blk):
            r1 = min(n, r0 + blk)
            drop = rng.integers(0, 2**32, size=(r1 - r0, n), dtype=np.uint32) >= thr
            R[r0:r1][drop] = 0
            del drop
    # mirror the upper triangle onto the lower one in place, one cache-sized tile pair at a time
    t = 1024
    for b0 in range(0, n, t):
        b1 = min(n, b0 + t)
        D = R[b0:b1, b0:b1]
        D[...] = np.triu(D) + np.triu(D, 1).T          # disjoint supports: no int8 overflow
        for c0 in range(b1, n, t):
            c1 = min(n, c0 + t)
            R[c0:c1, b0:b1] = R[b0:b1, c0:c1].T
    c = np.diagonal(R).astype(np.int32).copy()
    np.fill_diagonal(R, 0)
    Q = R if np.dtype(dtype) == np.int8 else R.astype(dtype)
    return Q, c


def heterogeneous_shapes(count: int, seed: int = 0, n_lo: int = 500, n_hi: int = 20000, dens_lo: float = 0.01,
                         dens_hi: float = 1.0):
    """(n_k, density_k) of the ``count`` instances of a heterogeneous batch: n ~ U{n_lo..n_hi},
    density ~ U[dens_lo, dens_hi]."""
    rng = _rng(seed, _TAG_HETERO)
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = float(rng.uniform(dens_lo, dens_hi))
        out.append((n, d))
    return out


def heterogeneous_qubo(k: int, count: int, seed: int = 0, n_lo: int = 500, n_hi: int = 20000,
                       dens_lo: float = 0.01, dens_hi: float = 1.0, lo: int = -100, hi: int = 100, dtype=np.int32):
    """Instance k of a heterogeneous batch (``dense_qubo`` at the k-th drawn size and density), from
    a generator of its own, so that instances can be drawn independently of one another (in
    parallel, or one at a time)."""
    n, d = heterogeneous_shapes(count, seed, n_lo, n_hi, dens_lo, dens_hi)[k]
    rng = np.random.Generator(np.random.PCG64([int(seed) & (2**63 - 1), _TAG_HETERO, 1 + int(k)]))
    return dense_qubo(n, lo=lo, hi=hi, density=d, rng=rng, dtype=dtype)


def iter_heterogeneous_qubos(count: int, seed: int = 0, n_lo: int = 500, n_hi: int = 20000,
                             dens_lo: float = 0.01, dens_hi: float = 1.0, lo: int = -100, hi: int = 100):
    """Yield the ``count`` dense QUBOs ``(Q, c)`` of a heterogeneous batch one at a time (at
    n_hi = 20,000 the whole batch is ~35 GB of int32 on the host)."""
    for k in range(count):
        yield heterogeneous_qubo(k, count, seed, n_lo, n_hi, dens_lo, dens_hi, lo, hi)


def heterogeneous_qubos(count: int, seed: int = 0, n_lo: int = 500, n_hi: int = 20000,
                        dens_lo: float = 0.01, dens_hi: float = 1.0, lo: int = -100, hi: int = 100):
    """The same instances as ``iter_heterogeneous_qubos``, as a list."""
    return list(iter_heterogeneous_qubos(count, seed, n_lo, n_hi, dens_lo, dens_hi, lo, hi))


# ----------------------------------------------------------------------------------------
# graphs (edge lists with i < j) and their CSR / QUBO forms
# ----------------------------------------------------------------------------------------
def _pm1(rng, m):
    return np.where(rng.integers(0, 2, size=m) == 1, 1, -1).astype(np.int32)


def maxcut_er(n: int, mean_degree: float = 6.0, seed: int = 0, weights: str = "pm1"):
    """Erdos-Renyi G(n, p) with p = mean_degree/(n-1); weights +-1 (or 1). Returns (i, j, w)."""
    rng = _rng(seed, _TAG_ER)
    p = mean_degree / (n - 1)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < p
    i, j = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    w = _pm1(rng, i.size) if weights == "pm1" else np.ones(i.size, np.int32)
    return i, j, w


def maxcut_torus(rows: int = 100, cols: int = 100, seed: int = 0, weights: str = "pm1"):
    """Periodic rows x cols grid (4 neighbours per vertex, 2*rows*cols edges)."""
    rng = _rng(seed, _TAG_TORUS)
    v = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    right = np.roll(v, -1, axis=1)
    down = np.roll(v, -1, axis=0)
    a = np.concatenate([v.ravel(), v.ravel()])
    b = np.concatenate([right.ravel(), down.ravel()])
    i = np.minimum(a, b).astype(np.int32)
    j = np.maximum(a, b).astype(np.int32)
    w = _pm1(rng, i.size) if weights == "pm1" else np.ones(i.size, np.int32)
    return i, j, w


def _switch_repair(a, b, n, rng, max_steps=None):
    """Remove loops and multi-edges from a pairing by random edge switches: a bad edge (u, v) and a
    random edge (w, z) become (u, w), (v, z) when neither new edge is a loop or already present."""
    a, b = a.copy(), b.copy()
    m = a.size
    cnt = {}

    def key(u, v):
        return (u, v) if u < v else (v, u)

    for k in range(m):
        kk = key(a[k], b[k])
        cnt[kk] = cnt.get(kk, 0) + 1

    def is_bad(k):
        return a[k] == b[k] or cnt[key(a[k], b[k])] > 1

    bad = [k for k in range(m) if is_bad(k)]
    steps = 0
    limit = max_steps if max_steps is not None else 200 * m
    while bad:
        steps += 1
        if steps > limit:
            raise RuntimeError("edge switching did not converge")
        k = bad[-1]
        if not is_bad(k):
            bad.pop()
            continue
        q = int(rng.integers(0, m))
        if q == k:
            continue
        u, v, w, z = a[k], b[k], a[q], b[q]
        e1, e2 = key(u, w), key(v, z)
        if u == w or v == z or e1 == e2:
            continue
        cnt[key(u, v)] -= 1
        cnt[key(w, z)] -= 1
        if cnt.get(e1, 0) or cnt.get(e2, 0):
            cnt[key(u, v)] += 1
            cnt[key(w, z)] += 1
            continue
        a[k], b[k], a[q], b[q] = u, w, v, z
        cnt[e1] = cnt.get(e1, 0) + 1
        cnt[e2] = cnt.get(e2, 0) + 1
        bad.pop()
    return a, b


def _regular_edges(n: int, d: int, rng: np.random.Generator, max_tries: int = 200):
    """Random simple d-regular graph: pairing model, rejecting loops and multi-edges; when
    rejection is hopeless (large d), one pairing repaired by random edge switches."""
    if (n * d) % 2:
        raise ValueError("n*d must be even")
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    if d > 8:
        perm = rng.permutation(stubs)
        a, b = _switch_repair(perm[0::2], perm[1::2], n, rng)
        lo_, hi_ = np.minimum(a, b), np.maximum(a, b)
        order = np.argsort(lo_ * n + hi_)
        return lo_[order].astype(np.int32), hi_[order].astype(np.int32)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        a, b = perm[0::2], perm[1::2]
        if np.any(a == b):
            continue
        lo_, hi_ = np.minimum(a, b), np.maximum(a, b)
        key = lo_ * n + hi_
        if np.unique(key).size != key.size:
            continue
        order = np.argsort(key)
        return lo_[order].astype(np.int32), hi_[order].astype(np.int32)
    raise RuntimeError("pairing model did not produce a simple graph")


def maxcut_regular(n: int = 20000, d: int = 4, seed: int = 0, weights: str = "unit"):
    """Random d-regular graph (pairing model with rejection); unit weights by default."""
    rng = _rng(seed, _TAG_REGULAR)
    i, j = _regular_edges(n, d, rng)
    w = _pm1(rng, i.size) if weights == "pm1" else np.ones(i.size, np.int32)
    return i, j, w


def csr_from_edges(n: int, i, j, w):
    """Symmetric CSR (both directions, columns sorted within a row) of the edge list."""
    rows = np.concatenate([i, j]).astype(np.int64)
    cols = np.concatenate([j, i]).astype(np.int64)
    vals = np.concatenate([w, w]).astype(np.int32)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), vals


def maxcut_qubo(n: int, i, j, w):
    """Max-Cut as QUBO: ``Q = W`` in CSR (both directions) and ``c = -W 1``."""
    rowptr, col, val = csr_from_edges(n, i, j, w)
    c = np.zeros(n, dtype=np.int64)
    np.add.at(c, i, w)
    np.add.at(c, j, w)
    return rowptr, col, val, (-c).astype(np.int32)


def mis_regular(n: int, d: int, seed: int = 0, lam: int = 4):
    """MIS on a random d-regular graph as QUBO: CSR ``Q`` (lam/2 both ways) and ``c = -1``."""
    if lam % 2:
        raise ValueError("lam must be even so that Q stays integral")
    rng = _rng(seed, _TAG_MIS)
    i, j = _regular_edges(n, d, rng)
    rowptr, col, val = csr_from_edges(n, i, j, np.full(i.size, lam // 2, np.int32))
    return rowptr, col, val, -np.ones(n, dtype=np.int32), (i, j)


def dense_from_csr(n: int, rowptr, col, val):
    """Dense int32 copy of a CSR matrix (small n only)."""
    Q = np.zeros((n, n), dtype=np.int32)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    np.add.at(Q, (rows, col), val)
    return Q


# ----------------------------------------------------------------------------------------
# hyper-parameters
# ----------------------------------------------------------------------------------------
@dataclasses.dataclass
class GdaParams:
    """Hyper-parameters of one batched PDBO run (names follow Algorithm 1 and App. C)."""
    restarts: int          # B
    iters: int             # T_max
    alpha: float           # primal step
    beta: float            # dual step
    ybar: float            # y^0 = ybar * 1
    delta: float = 0.01    # tolerance of the perturbation rule (value not given in the paper)
    grad_tol: float = 0.02  # gradient threshold of the perturbation rule (2*delta in Alg. 1)
    eval_every: int = 10   # K: rounding + exact objective every K iterations and at T
    seed: int = 0

    def asdict(self):
        return dataclasses.asdict(self)


def graph_params(kind: str = "maxcut", restarts: int = 100, iters: int = 1000,
                 delta: float = 0.01, eval_every: int = 10, seed: int = 0) -> GdaParams:
    """The paper's hyper-parameter table (App. C.1): Max-Cut ybar=6, alpha=beta=0.025;
    MIS ybar=5, alpha=beta=0.02; the gradient threshold is 2*delta as in Algorithm 1."""
    table = {"maxcut": (6.0, 0.025, 0.025), "mis": (5.0, 0.02, 0.02)}
    ybar, a, b = table[kind]
    return GdaParams(restarts=restarts, iters=iters, alpha=a, beta=b, ybar=ybar, delta=delta,
                     grad_tol=2 * delta, eval_every=eval_every, seed=seed)


def spectral_scale(Q) -> float:
    """Semicircle estimate of |lambda_min| of the symmetric part of Q (zero diagonal):
    2 * ||Q_sym||_F / sqrt(n), with Q_sym = (Q + Q^T)/2 off the diagonal."""
    Q = np.asarray(Q)
    n = Q.shape[0]
    ss = 0.0
    blk = 1024
    for r0 in range(0, n, blk):
        r1 = min(n, r0 + blk)
        S = Q[r0:r1].astype(np.float64) + Q[:, r0:r1].T.astype(np.float64)
        S[np.arange(r1 - r0), np.arange(r0, r1)] = 0.0
        ss += float(np.sum(S * S)) * 0.25
    return 2.0 * math.sqrt(ss) / math.sqrt(n)


def csr_spectral_scale(n: int, rowptr, col, val) -> float:
    """spectral_scale of a CSR Q: 2 ||Q_sym||_F / sqrt(n) (off-diagonal part)."""
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr)))
    col = np.asarray(col)
    off = rows != col
    sym = {}
    for r, cc, v in zip(rows[off], col[off], np.asarray(val)[off]):
        k = (r, cc) if r < cc else (cc, r)
        sym[k] = sym.get(k, 0) + int(v)
    ss = sum(2 * (0.5 * v) ** 2 for v in sym.values())
    return 2.0 * math.sqrt(ss) / math.sqrt(n)


def dense_params(Q, restarts: int, iters: int, delta: float = 0.01, eval_every: int = 50,
                 seed: int = 0, lam_hat: float | None = None) -> GdaParams:
    """Hyper-parameters for dense integer QUBO, carried over from the paper's Max-Cut regime.

    The paper tunes (ybar, alpha, beta) for graphs only.  The map
    (A, c', ybar, alpha, beta, tol) -> (sA, sc', s ybar, alpha/s, s beta, s tol) leaves every
    primal iterate unchanged, so with s = lam_hat/4 (lam_hat estimating |lambda_min|) the
    Max-Cut values ybar=6, alpha=beta=0.025 keep ybar at 1.5x |lambda_min|, i.e. the convex
    start of the landscape analysis (section 4.4)."""
    lam = spectral_scale(Q) if lam_hat is None else lam_hat
    lam = max(lam, 1.0)              # an (almost) empty Q keeps finite steps
    s = lam / 4.0
    return GdaParams(restarts=restarts, iters=iters, alpha=0.025 / s, beta=0.025 * s,
                     ybar=6.0 * s, delta=delta, grad_tol=2 * delta * s, eval_every=eval_every,
                     seed=seed)
