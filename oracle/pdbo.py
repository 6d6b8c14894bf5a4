"""FP64 CPU oracle of PDBO's batched primal-dual GDA (arXiv 2509.21064).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or run this module.  The product package
(``paper_2509_21064_gb300``) never imports it and shares no code with it; the two meet only
through the seeded inputs of ``workloads/``.

It is plain and slow on purpose: numpy float64 (int64 for objectives), one library matmul per
contraction, no blocking, fusion or reordering beyond what each cited passage states.  Batched
arrays are restart-major: ``X[r, i]`` is coordinate i of restart r.

Functions and what pins them (tests/test_oracle_*.py, tests/golden/):

==================  ===============================================  ===========================
function            follows                                          pinned by
==================  ===============================================  ===========================
canonicalize        Prop. 2.4 (exponents dropped on binary points)   Def. 2.2 expectation by
 (and _csr)                                                          enumeration; golden file;
                                                                     dense == CSR form
objective           Eq. 1 with the QUBO objective                    Max-Cut edge count; MIS
                                                                     count; golden file
multilinear         Def. 2.2 / Prop. 2.4 closed form                 enumeration; Lemma 2.3
lagrangian          Lagrangian of section 3.1, g(x) = x^2 - x or     Prop. 3.1 (L = F on binary
                    the entropy x log x + (1-x) log(1-x)             points); central finite
                                                                     differences; Example in 3.2;
                                                                     entropy: its three
                                                                     conditions of section 3.1
splitmix64/uniform  x^0 ~ Uniform([0,1]^n) (App. C.1) drawn from the  published SplitMix64 output
                    SplitMix64 generator (Steele, Lea, Flood 2014)   for seed 0
gda_step            Eq. 5 and Algorithm 1                            hand-worked golden steps;
                                                                     box, monotone-dual and
                                                                     telescoping invariants;
                                                                     Prop. 3.3 bound; convex
                                                                     special case (KKT)
lagrangian_single   single-constraint Lagrangian of the PDBO-s        central finite differences;
                    variant (section 4, Discussion and ablation):    L = F on binary points
                    f(x) + mu sum_i g(x_i), one dual per restart
gda_step_single     Algorithm 1 on that Lagrangian                   beta = 0 reduces it to
                                                                     gda_step exactly; on a
                                                                     symmetric instance it is
                                                                     gda_step with beta / n
certificate         dual bound of the section on the dual            equals L at the box
                    certificate: L(x) + min over the box of          minimiser (scipy L-BFGS-B);
                    <grad L(x), z - x>, valid when L(., ybar) is     below brute-force min F
                    convex on the box
round_bits / run    best-of-B retention (section 4.2), evaluation    brute force over 2^n;
                    every K iterations and at T                      tie rules on tiny inputs
brute_force         Lemma 2.3 (min over the vertices)                exhaustive by definition
==================  ===============================================  ===========================

Parity unpinned: none of the above.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


# ----------------------------------------------------------------------------------------
# problem and its multilinear extension
# ----------------------------------------------------------------------------------------
def canonicalize(Q, c=None):
    """Multilinear form of ``F(x) = x^T Q x + c^T x`` (Prop. 2.4).

    On binary points x_i^2 = x_i, so the diagonal of Q moves into the linear term and each
    off-diagonal pair (i, j), (j, i) becomes one bilinear term:
    ``f(x) = 1/2 x^T A x + c'^T x`` with ``A_ij = Q_ij + Q_ji`` (i != j), ``A_ii = 0`` and
    ``c'_i = c_i + Q_ii``.  Returns (A, c') in float64.
    """
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[0]
    c = np.zeros(n) if c is None else np.asarray(c, dtype=np.float64)
    A = Q + Q.T
    np.fill_diagonal(A, 0.0)
    cp = c + np.diagonal(Q)
    return A, cp


def canonicalize_csr(n, rowptr, col, val, c=None):
    """Prop. 2.4 for a CSR Q: the same multilinear form as ``canonicalize``, as a scipy sparse A
    (A = Q + Q^T off the diagonal, c' = c + diag Q).  scipy is only the storage and the matmul."""
    import scipy.sparse as sp
    Qs = sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(col), np.asarray(rowptr)), shape=(n, n))
    diag = Qs.diagonal()
    A = (Qs + Qs.T).tolil()
    A.setdiag(0.0)
    A = A.tocsr()
    A.eliminate_zeros()
    c = np.zeros(n) if c is None else np.asarray(c, dtype=np.float64)
    return A, c + diag


def objective(Q, c, b):
    """Exact ``F(b) = b^T Q b + c^T b`` for one binary vector (Eq. 1, QUBO), as a Python int."""
    Q = np.asarray(Q, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    c = np.zeros(Q.shape[0], np.int64) if c is None else np.asarray(c, dtype=np.int64)
    return int(b @ (Q @ b)) + int(c @ b)


def objective_batch(Q, c, Bits):
    """Exact F (Eq. 1, QUBO) for every row of ``Bits`` (B x n, values 0/1) in int64."""
    Q = np.asarray(Q, dtype=np.int64)
    Bm = np.asarray(Bits, dtype=np.int64)
    c = np.zeros(Q.shape[0], np.int64) if c is None else np.asarray(c, dtype=np.int64)
    return np.einsum("ri,ri->r", Bm @ Q.T, Bm) + Bm @ c


def objective_csr(n, rowptr, col, val, c, b):
    """Exact F(b) (Eq. 1, QUBO) for a CSR Q: sum over stored (i, j, q) of q b_i b_j, plus c^T b."""
    b = np.asarray(b, dtype=np.int64)
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr)))
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.int64)
    c = np.zeros(n, np.int64) if c is None else np.asarray(c, dtype=np.int64)
    return int(np.sum(val * b[rows] * b[col])) + int(c @ b)


def multilinear(A, cp, x):
    """Closed form of the multilinear extension (Def. 2.2, Prop. 2.4), ``f(x) = 1/2 x^T A x + c'^T x``."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x @ (A @ x) + cp @ x


# ----------------------------------------------------------------------------------------
# Lagrangian (section 3.1) with g(x) = x^2 - x (section 4.2)
# ----------------------------------------------------------------------------------------
def g(x):
    """Binarity constraint function g(x) = x^2 - x of section 4.2 (zero exactly at 0 and 1)."""
    return x * x - x


def g_prime(x):
    """g'(x) = 2x - 1 (section 4.2's g), the y-weighted term of dL/dx in Algorithm 1."""
    return 2.0 * x - 1.0


ENTROPY_EPS = 1e-6


def g_entropy(x):
    """The entropy constraint function x log x + (1 - x) log(1 - x) named in section 3.1, extended
    continuously by g(0) = g(1) = 0."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(x > 0.0, x * np.log(np.where(x > 0.0, x, 1.0)), 0.0)
        b = np.where(x < 1.0, (1.0 - x) * np.log(np.where(x < 1.0, 1.0 - x, 1.0)), 0.0)
    return a + b


def g_entropy_prime(x):
    """Derivative of the entropy g of section 3.1, log(x / (1 - x)), unbounded at 0 and 1: taken at
    x clamped to [ENTROPY_EPS, 1 - ENTROPY_EPS]."""
    xc = np.clip(np.asarray(x, dtype=np.float64), ENTROPY_EPS, 1.0 - ENTROPY_EPS)
    return np.log(xc) - np.log1p(-xc)


def _g_pair(kind):
    if kind == "quadratic":
        return g, g_prime
    if kind == "entropy":
        return g_entropy, g_entropy_prime
    raise ValueError("g must be 'quadratic' or 'entropy'")


def lagrangian(A, cp, X, Y, gkind="quadratic"):
    """Value and gradients of ``L(x, y) = f(x) + sum_i y_i g(x_i)`` for every restart.

    Returns ``(L[B], dL/dX [B, n], dL/dY [B, n])`` with
    ``dL/dx = A x + c' + y * g'(x)`` and ``dL/dy = g(x)``; ``gkind`` selects g (section 3.1).
    """
    gf, gp = _g_pair(gkind)
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    AX = np.asarray((A @ X.T).T)          # A dense or scipy sparse
    Lval = 0.5 * np.einsum("ri,ri->r", X, AX) + X @ cp + np.sum(Y * gf(X), axis=1)
    GX = AX + cp[None, :] + Y * gp(X)
    GY = gf(X)
    return Lval, GX, GY


def lagrangian_single(A, cp, X, MU):
    """Single-constraint variant (PDBO-s, section 4 Discussion): the constraint sum_i g(x_i) = 0
    with one dual mu per restart, ``L_s(x, mu) = f(x) + mu * sum_i g(x_i)``.

    Returns ``(L[B], dL/dX [B, n], dL/dmu [B])`` with ``dL/dx = A x + c' + mu g'(x)`` and
    ``dL/dmu = sum_i g(x_i)``.
    """
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    MU = np.asarray(MU, dtype=np.float64).reshape(-1)
    AX = np.asarray((A @ X.T).T)
    G = g(X)
    Lval = 0.5 * np.einsum("ri,ri->r", X, AX) + X @ cp + MU * np.sum(G, axis=1)
    GX = AX + cp[None, :] + MU[:, None] * g_prime(X)
    GMU = np.sum(G, axis=1)
    return Lval, GX, GMU


# ----------------------------------------------------------------------------------------
# x^0 ~ Uniform([0,1]^n): SplitMix64 as a counter-based generator
# ----------------------------------------------------------------------------------------
def splitmix64_mix(z):
    """SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014) on uint64 numpy arrays."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix64_stream(seed, k):
    """Output number ``k`` (0-based) of SplitMix64 seeded with ``seed``: mix(seed + (k+1)*gamma)."""
    seed = np.uint64(int(seed) & MASK64)
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = seed + (k + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
    return splitmix64_mix(state)


def uniform24(seed, r, i):
    """U(seed, r, i) in [0, 1): top 24 bits of stream output number r * 2^32 + i, times 2^-24.

    Exactly representable in float32, so the GPU and this oracle start from identical x^0."""
    r = np.asarray(r, dtype=np.uint64)
    i = np.asarray(i, dtype=np.uint64)
    k = (r << np.uint64(32)) | i
    z = splitmix64_stream(seed, k)
    return (z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def init_state(n, B, seed, ybar):
    """x^0_{r,i} = U(seed, r, i); y^0 = ybar * 1 (App. C.1)."""
    r = np.arange(B, dtype=np.uint64)[:, None]
    i = np.arange(n, dtype=np.uint64)[None, :]
    X0 = uniform24(seed, r, i)
    Y0 = np.full((B, n), float(ybar))
    return X0, Y0


# ----------------------------------------------------------------------------------------
# one iteration of Algorithm 1 for every restart
# ----------------------------------------------------------------------------------------
def gda_step(A, cp, X, Y, alpha, beta, delta, grad_tol=None, gkind="quadratic"):
    """One simultaneous projected GDA iteration with the delta-perturbation (Algorithm 1).

    For each restart and coordinate i, with d_i = dL/dx_i (x^t, y^t):
      if |x_i - 1/2| <= delta and |d_i| <= grad_tol and y_i <= 0:
          x_i <- 1/2 - delta if x_i <= 1/2 else 1/2 + delta
      else:
          x_i <- Pi_[0,1](x_i - alpha d_i)
      y_i <- y_i + beta g(x_i)       (g evaluated at the old x_i: the updates are simultaneous)
    ``grad_tol`` defaults to 2*delta, the threshold Algorithm 1 prints; ``gkind`` selects g.
    Returns (X^{t+1}, Y^{t+1}, D^t).
    """
    if grad_tol is None:
        grad_tol = 2.0 * delta
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    _, D, GY = lagrangian(A, cp, X, Y, gkind)
    stagnating = (np.abs(X - 0.5) <= delta) & (np.abs(D) <= grad_tol) & (Y <= 0.0)
    perturbed = np.where(X <= 0.5, 0.5 - delta, 0.5 + delta)
    projected = np.minimum(1.0, np.maximum(0.0, X - alpha * D))
    Xn = np.where(stagnating, perturbed, projected)
    Yn = Y + beta * GY
    return Xn, Yn, D


def gda_step_single(A, cp, X, MU, alpha, beta, delta, grad_tol=None):
    """Algorithm 1 applied to the single-constraint Lagrangian (PDBO-s): the same primal step and
    delta-perturbation with the restart's one dual mu in place of y_i, and the dual ascent
    mu <- mu + beta * sum_i g(x_i) on the old x (simultaneous updates).
    Returns (X^{t+1}, MU^{t+1}, D^t)."""
    if grad_tol is None:
        grad_tol = 2.0 * delta
    X = np.asarray(X, dtype=np.float64)
    MU = np.asarray(MU, dtype=np.float64).reshape(-1)
    _, D, GMU = lagrangian_single(A, cp, X, MU)
    stagnating = (np.abs(X - 0.5) <= delta) & (np.abs(D) <= grad_tol) & (MU[:, None] <= 0.0)
    perturbed = np.where(X <= 0.5, 0.5 - delta, 0.5 + delta)
    projected = np.minimum(1.0, np.maximum(0.0, X - alpha * D))
    Xn = np.where(stagnating, perturbed, projected)
    MUn = MU + beta * GMU
    return Xn, MUn, D


def certificate(A, cp, ybar, x):
    """Dual certificate (section on the dual certificate): with y = ybar * 1 and L(., y) convex on
    the box, every box point x gives min F >= min_box L(., y) >= L(x) + min_{z in box} <grad L(x),
    z - x> = L(x) - sum_i (grad_i x_i - min(0, grad_i)).  Returns that bound."""
    x = np.asarray(x, dtype=np.float64).reshape(1, -1)
    L, GX, _ = lagrangian(A, cp, x, np.full_like(x, float(ybar)))
    gr = GX[0]
    return float(L[0] - np.sum(gr * x[0] - np.minimum(0.0, gr)))


def round_bits(X):
    """Rounding of section 4.2: b_i = [x_i > 1/2] for each restart (ties go to 0, the x <= 1/2 side)."""
    return (np.asarray(X) > 0.5).astype(np.uint8)


def eval_points(T, K):
    """Iteration counts t at which candidates are evaluated (best retention of section 4.2, on
    the schedule this implementation reads into it): K, 2K, ... and T (never t=0)."""
    pts = list(range(K, T + 1, K))
    if T > 0 and (not pts or pts[-1] != T):
        pts.append(T)
    return pts


def run(Q, c, restarts, iters, alpha, beta, ybar, delta=0.01, grad_tol=None, eval_every=10,
        seed=0, X0=None, Y0=None, dump_iters=0, A=None, cp=None, dual="coordinate", gkind="quadratic",
        **_ignored):
    """Batched PDBO: B restarts of Algorithm 1, best candidate retained (section 4.2).

    Candidates b = round_bits(x^t) are evaluated exactly at every t in eval_points(T, K).
    Per restart the best F is kept with its earliest t (strict improvement only); the global
    best is the lexicographic minimum of (F, t, r).  ``dump_iters`` keeps (x, y, d) for the
    first iterations (parity dumps).  ``dual="single"`` runs the PDBO-s variant
    (``gda_step_single``): Y is then one dual per restart, shape (B,).
    """
    Q = np.asarray(Q)
    n = Q.shape[0]
    if A is None or cp is None:
        A, cp = canonicalize(Q, c)
    if dual not in ("coordinate", "single"):
        raise ValueError("dual must be 'coordinate' or 'single'")
    if dual == "single":
        Y0 = np.full(restarts, float(ybar)) if Y0 is None else np.asarray(Y0, dtype=np.float64).reshape(-1)
    if X0 is None:
        X0, Y0d = init_state(n, restarts, seed, ybar)
        if Y0 is None:
            Y0 = Y0d
    if Y0 is None:
        Y0 = np.full((restarts, n), float(ybar))
    X = np.array(X0, dtype=np.float64)
    Y = np.array(Y0, dtype=np.float64)
    if dual == "single":
        step = gda_step_single
    else:
        def step(A_, cp_, X_, Y_, a_, b_, d_, gt_):
            return gda_step(A_, cp_, X_, Y_, a_, b_, d_, gt_, gkind)
    pts = set(eval_points(iters, eval_every))
    best_F = np.full(restarts, np.iinfo(np.int64).max, dtype=np.int64)
    best_t = np.full(restarts, -1, dtype=np.int64)
    best_bits = np.zeros((restarts, n), dtype=np.uint8)
    evals = []
    dumps = {"x": [X.copy()], "y": [Y.copy()], "d": []}
    for t in range(iters):
        Xn, Yn, D = step(A, cp, X, Y, alpha, beta, delta, grad_tol)
        if t < dump_iters:
            dumps["d"].append(D)
            dumps["x"].append(Xn.copy())
            dumps["y"].append(Yn.copy())
        X, Y = Xn, Yn
        tt = t + 1
        if tt in pts:
            bits = round_bits(X)
            F = objective_batch(Q, c, bits)
            evals.append((tt, F.copy()))
            better = F < best_F
            best_F[better] = F[better]
            best_t[better] = tt
            best_bits[better] = bits[better]
    out = {"X": X, "Y": Y, "best_F": best_F, "best_t": best_t, "best_bits": best_bits,
           "evals": evals, "dumps": dumps}
    if iters > 0:
        order = np.lexsort((np.arange(restarts), best_t, best_F))
        r = int(order[0])
        out.update(F_star=int(best_F[r]), t_star=int(best_t[r]), r_star=r,
                   x_star=best_bits[r].copy())
    return out


# ----------------------------------------------------------------------------------------
# exhaustive minimum (Lemma 2.3: the minimum over the box is attained at a vertex)
# ----------------------------------------------------------------------------------------
def brute_force(Q, c, chunk=1 << 15):
    """min F over all 2^n binary points (n <= 24; Lemma 2.3: the box minimum is attained there),
    and every minimiser (as an array of ints)."""
    Q = np.asarray(Q, dtype=np.int64)
    n = Q.shape[0]
    if n > 24:
        raise ValueError("brute force limited to n <= 24")
    c = np.zeros(n, np.int64) if c is None else np.asarray(c, dtype=np.int64)
    shifts = np.arange(n, dtype=np.int64)
    best = None
    arg = []
    for s in range(0, 1 << n, chunk):
        idx = np.arange(s, min(1 << n, s + chunk), dtype=np.int64)
        Bm = (idx[:, None] >> shifts[None, :]) & 1
        F = np.einsum("ki,ki->k", Bm @ Q.T, Bm) + Bm @ c
        m = int(F.min())
        if best is None or m < best:
            best, arg = m, list(idx[F == m])
        elif m == best:
            arg.extend(idx[F == m])
    return best, np.array(arg, dtype=np.int64)


def bits_of(index, n):
    """Binary vector (uint8, length n) of an enumeration index used by ``brute_force``."""
    return ((int(index) >> np.arange(n)) & 1).astype(np.uint8)
