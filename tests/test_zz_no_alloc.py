"""sbo_lagrangian_noalloc against sbo_lagrangian, through the C ABI.

The allocation-free entry point exists for callers that may not call cudaMalloc (processes whose
device memory belongs to a framework's pool or a fixed budget, loops that cannot absorb an
allocation's implicit synchronisation).  It must give the same values and gradients as the
allocating entry point, call after call, even though every call reuses the same fixed scratch
array, also when consecutive calls come from problems of different sizes; and those values are
checked against the FP64 oracle's Lagrangian.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the FP32 tolerance of the parity tests; both calls run the same arithmetic


def _normwise(a, b):
    num = np.max(np.abs(a - b), axis=-1)
    den = np.maximum(np.max(np.abs(b), axis=-1), 1e-30)
    return float(np.max(num / den))


@pytest.mark.parametrize("prec", [S.SBO_BF16, S.SBO_FP32])
def test_noalloc_matches_allocating_entry_point_twice_in_a_row(prec):
    import torch
    build_lib()
    n, B = 777, 96
    Q, c = W.dense_qubo(n, seed=21)
    rng = np.random.default_rng(5)
    stream = torch.cuda.current_stream()
    with S.Problem.dense(Q, c, precision=prec) as P:
        for call in range(2):                 # two calls in a row share the scratch array
            X = torch.tensor(rng.random((B, n)), dtype=torch.float32, device="cuda")
            Y = torch.tensor(rng.normal(scale=30.0, size=(B, n)), dtype=torch.float32, device="cuda")
            g = torch.tensor(rng.normal(size=B), dtype=torch.float32, device="cuda")
            outs = []
            for fn in (S.sbo_lagrangian, S.sbo_lagrangian_noalloc):
                L = torch.empty(B, device="cuda")
                GX = torch.empty_like(X)
                GY = torch.empty_like(X)
                fn(P.h, B, X.data_ptr(), Y.data_ptr(), g.data_ptr(), L.data_ptr(), GX.data_ptr(), GY.data_ptr(),
                   stream)
                torch.cuda.synchronize()
                outs.append((L.cpu().numpy(), GX.cpu().numpy(), GY.cpu().numpy()))
            (L0, GX0, GY0), (L1, GX1, GY1) = outs
            assert _normwise(GX1, GX0) <= TOL, call
            assert _normwise(GY1, GY0) <= TOL, call
            # L sums per-tile partials with float atomics in no fixed order: compare normwise over
            # the batch, like every other vector in these tests
            assert np.max(np.abs(L1 - L0)) / np.max(np.abs(L0)) <= TOL, call


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    build_lib()
    n = 2000
    Q = np.zeros((n, n), dtype=np.int32)
    B = 5000                                    # 5000 * 2000 * 2 bytes > 16 MiB
    X = torch.zeros(1, device="cuda")
    with S.Problem.dense(Q, None, precision=S.SBO_BF16) as P:
        with pytest.raises(S.SboError) as e:
            S.sbo_lagrangian_noalloc(P.h, B, X.data_ptr(), X.data_ptr(), None, None, None, None, None)
        assert e.value.status == S.SBO_EINVAL
        assert "scratch" in e.value.message


def _lagr(fn, P, X, Y, g):
    import torch
    B = X.shape[0]
    L = torch.empty(B, device="cuda")
    GX = torch.empty_like(X)
    GY = torch.empty_like(X)
    fn(P.h, B, X.data_ptr(), Y.data_ptr(), g.data_ptr(), L.data_ptr(), GX.data_ptr(), GY.data_ptr(),
       torch.cuda.current_stream())
    torch.cuda.synchronize()
    return L.cpu().numpy(), GX.cpu().numpy(), GY.cpu().numpy()


def test_noalloc_alternating_problem_sizes():
    """Calls alternate between problems of n = 1000 and n = 777 (row pitches 1000 and 784 in the
    shared scratch): each call's result matches the allocating entry point's, whatever the
    previous call left in the scratch."""
    import torch
    build_lib()
    rng = np.random.default_rng(8)
    probs = []
    for n in (1000, 777):
        Q, c = W.dense_qubo(n, seed=n)
        probs.append(S.Problem.dense(Q, c, precision=S.SBO_BF16))
    try:
        for rnd in range(2):
            for P, B in zip(probs, (120, 96)):
                X = torch.tensor(rng.random((B, P.n)), dtype=torch.float32, device="cuda")
                Y = torch.tensor(rng.normal(scale=30.0, size=(B, P.n)), dtype=torch.float32, device="cuda")
                g = torch.ones(B, device="cuda")
                L0, GX0, GY0 = _lagr(S.sbo_lagrangian, P, X, Y, g)
                L1, GX1, GY1 = _lagr(S.sbo_lagrangian_noalloc, P, X, Y, g)
                assert _normwise(GX1, GX0) <= TOL and _normwise(GY1, GY0) <= TOL, (rnd, P.n)
                assert np.max(np.abs(L1 - L0)) / np.max(np.abs(L0)) <= TOL, (rnd, P.n)
    finally:
        for P in probs:
            P.close()


@pytest.mark.parametrize("prec", [S.SBO_BF16, S.SBO_FP32])
def test_noalloc_against_the_oracle(prec):
    """Value and gradients against the FP64 oracle's Lagrangian (section 3.1), whose gradient is
    pinned to central differences.  x on a 1/256 grid is exact in BF16, so only FP32 accumulation
    separates the two on either precision: 1e-5 for dL/dx and L, 1e-6 for dL/dy = g(x)."""
    import torch
    build_lib()
    n, B = 900, 64
    Q, c = W.dense_qubo(n, seed=4)
    A, cp = O.canonicalize(Q, c)
    rng = np.random.default_rng(12)
    Xh = rng.integers(0, 257, size=(B, n)) / 256.0
    Yh = rng.normal(scale=40.0, size=(B, n)).astype(np.float32).astype(np.float64)
    gh = rng.normal(size=B).astype(np.float32).astype(np.float64)
    L_o, GX_o, GY_o = O.lagrangian(A, cp, Xh, Yh)
    with S.Problem.dense(Q, c, precision=prec) as P:
        X = torch.tensor(Xh, dtype=torch.float32, device="cuda")
        Y = torch.tensor(Yh, dtype=torch.float32, device="cuda")
        g = torch.tensor(gh, dtype=torch.float32, device="cuda")
        for call in range(2):
            L, GX, GY = _lagr(S.sbo_lagrangian_noalloc, P, X, Y, g)
            assert _normwise(GX, gh[:, None] * GX_o) <= 1e-5, call
            assert _normwise(GY, gh[:, None] * GY_o) <= 1e-6, call
            assert np.max(np.abs(L - L_o)) / np.max(np.abs(L_o)) <= 1e-5, call
