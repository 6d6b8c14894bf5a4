"""The dual certificate (sbo_dual_bound) and the sparse form of sbo_lagrangian, through the C ABI,
against the FP64 oracle."""
import numpy as np
import pytest
import scipy.optimize as so

import oracle as O
import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib
from _helpers import normwise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()
    S.lib()


def _box_min(A, cp, ybar):
    n = A.shape[0]
    fun = lambda x: float(O.lagrangian(A, cp, x[None, :], np.full((1, n), ybar))[0][0])
    jac = lambda x: O.lagrangian(A, cp, x[None, :], np.full((1, n), ybar))[1][0]
    res = so.minimize(fun, np.full(n, 0.5), jac=jac, method="L-BFGS-B", bounds=[(0.0, 1.0)] * n,
                      options={"ftol": 1e-15, "gtol": 1e-10, "maxiter": 50000})
    return res.x, res.fun


@pytest.mark.parametrize("n,prec", [(16, S.SBO_FP32), (16, S.SBO_BF16), (300, S.SBO_BF16), (300, S.SBO_FP32)])
def test_dense_dual_bound_is_valid_and_tight(n, prec):
    """ybar just above -lambda_min(A)/2 (A + 2 ybar I semidefinite): the bound lies below the
    brute-force minimum (n = 16), below L at the final point, and within 1e-4 of the oracle's
    certificate at scipy's box minimiser."""
    Q, c = W.dense_qubo(n, seed=n + 2)
    A, cp = O.canonicalize(Q, c)
    lam = np.linalg.eigvalsh(A)
    ybar = -lam.min() / 2.0 + 1e-3
    alpha = 1.0 / (lam.max() + 2.0 * ybar)
    with S.Problem.dense(Q, c, precision=prec) as P:
        lb, val = P.dual_bound(ybar, alpha, 20000)
    xs, Ls = _box_min(A, cp, ybar)
    cert = O.certificate(A, cp, ybar, xs)
    assert lb <= val + 1e-9
    assert abs(lb - cert) <= 1e-4 * max(1.0, abs(cert))
    if n <= 16:
        assert lb <= O.brute_force(Q, c)[0]


@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_FP8_E4M3])
def test_maxcut_dual_bound_caps_every_cut(prec):
    """20 x 20 +-1 torus: with ybar = -lambda_min(W) the certificate bounds every cut, including
    the best PDBO finds, and matches the oracle's certificate at the box minimiser."""
    import scipy.sparse.linalg as spla
    i, j, w = W.maxcut_torus(20, 20, seed=5)
    n = 400
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    A, cp = O.canonicalize_csr(n, rowptr, col, val, c)
    Ad = A.toarray()
    Wm = Ad / 2.0
    lam_w = float(np.linalg.eigvalsh(Wm).min())
    ybar = -lam_w + 1e-6
    alpha = 1.0 / (np.linalg.eigvalsh(Ad).max() + 2.0 * ybar)
    p = W.graph_params("maxcut", restarts=64, iters=2000, eval_every=10, seed=0)
    with S.Problem.csr(n, rowptr, col, val, c, precision=prec) as P:
        P.gda(S.params(**p.asdict()))
        x, F, _, _ = P.best()
        lb, val_ = P.dual_bound(ybar, alpha, 20000)
    cert = O.certificate(Ad, cp, ybar, _box_min(Ad, cp, ybar)[0])
    assert abs(lb - cert) <= 1e-4 * abs(cert)
    assert F >= lb                                   # -cut >= lower bound
    assert -lb >= int(np.sum(w * (x[i] != x[j])))


@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_BF16])
def test_csr_lagrangian_matches_the_oracle(prec):
    """The sparse Lagrangian (x on a 1/256 grid, exact in BF16): values and both gradients."""
    import torch
    n, B = 3001, 37
    i, j, w = W.maxcut_er(n, 6.0, seed=9)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    A, cp = O.canonicalize_csr(n, rowptr, col, val, c)
    rng = np.random.default_rng(1)
    X = rng.integers(0, 257, size=(B, n)) / 256.0
    Y = rng.normal(scale=10.0, size=(B, n)).astype(np.float32).astype(np.float64)
    gw = rng.normal(size=B).astype(np.float32).astype(np.float64)
    L_o, GX_o, GY_o = O.lagrangian(A, cp, X, Y)
    with S.Problem.csr(n, rowptr, col, val, c, precision=prec) as P:
        Xt = torch.tensor(X, dtype=torch.float32, device="cuda")
        Yt = torch.tensor(Y, dtype=torch.float32, device="cuda")
        gt = torch.tensor(gw, dtype=torch.float32, device="cuda")
        L = torch.empty(B, device="cuda")
        GX = torch.empty_like(Xt)
        GY = torch.empty_like(Xt)
        S.sbo_lagrangian(P.h, B, Xt.data_ptr(), Yt.data_ptr(), gt.data_ptr(), L.data_ptr(), GX.data_ptr(),
                         GY.data_ptr(), torch.cuda.current_stream())
        torch.cuda.synchronize()
    assert normwise(GX.cpu().numpy(), gw[:, None] * GX_o).max() <= 1e-5
    assert normwise(GY.cpu().numpy(), gw[:, None] * GY_o).max() <= 1e-6
    assert np.max(np.abs(L.cpu().numpy() - L_o)) / np.max(np.abs(L_o)) <= 1e-5
