"""sbo_create_dense_i8: an int8 Q builds the same canonical problem as its int32 copy (diagonal
and negative entries included): identical iterates, bests and evaluations on both precisions."""
import numpy as np
import pytest

import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib
from _helpers import to_gda_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_BF16])
def test_int8_and_int32_inputs_give_the_same_run(prec):
    build_lib()
    n = 777
    rng = np.random.default_rng(3)
    M = rng.integers(-128, 128, size=(n, n)).astype(np.int32)   # not symmetric, full int8 range
    c = rng.integers(-1000, 1000, size=n).astype(np.int32)
    p = W.dense_params(M, restarts=100, iters=60, eval_every=10, seed=2)
    prm = to_gda_params(p)
    out = []
    for Q in (M, M.astype(np.int8)):
        with S.Problem.dense(Q, c, precision=prec) as P:
            P.start(prm)
            P.run(60)
            X, Y = P.state()
            bits = rng.integers(0, 2, size=(5, n)).astype(np.uint8) if not out else out[0][3]
            out.append((X, Y, P.best(), bits, S.sbo_eval(P.h, bits)))
    (X1, Y1, b1, _, F1), (X2, Y2, b2, _, F2) = out
    assert np.array_equal(X1, X2) and np.array_equal(Y1, Y2)
    assert np.array_equal(b1[0], b2[0]) and b1[1:] == b2[1:]
    assert np.array_equal(F1, F2)


@pytest.mark.parametrize("n", [63, 65, 200, 333])
@pytest.mark.parametrize("qtype", [np.int32, np.int8])
@pytest.mark.parametrize("prec", [S.SBO_FP32, S.SBO_BF16])
def test_canonical_matrix_read_through_unit_points(n, qtype, prec):
    """The device's canonical form (Prop. 2.4: A = Q + Q^T with zero diagonal, c' = c + diag Q),
    read column by column: at x = e_k and y = 0 the Lagrangian's x-gradient is A e_k + c'.  Sizes
    below, at and across the 64-wide tiles of the canonicalisation, int32 and int8 inputs; every
    entry is exact in both storage types, so the comparison with the oracle's form is exact."""
    import torch
    import oracle.pdbo as O
    build_lib()
    rng = np.random.default_rng(n)
    M = rng.integers(-100, 101, size=(n, n)).astype(np.int32)
    c = rng.integers(-1000, 1000, size=n).astype(np.int32)
    A, cp = O.canonicalize(M, c)
    with S.Problem.dense(M.astype(qtype), c, precision=prec) as P:
        X = torch.eye(n, device="cuda", dtype=torch.float32)
        Y = torch.zeros(n, n, device="cuda")
        GX = torch.empty_like(X)
        S.sbo_lagrangian(P.h, n, X.data_ptr(), Y.data_ptr(), None, None, GX.data_ptr(), None,
                         torch.cuda.current_stream())
        torch.cuda.synchronize()
    got = GX.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, A.T + cp[None, :])


def test_int32_pair_sums_beyond_int32_are_rejected():
    """A_01 = Q_01 + Q_10 = 2^32 - 2 is formed in int64: the range check sees it (a 32-bit sum
    would wrap to -2 and pass)."""
    build_lib()
    Q = np.zeros((8, 8), np.int32)
    Q[0, 1] = Q[1, 0] = 2**31 - 1
    with pytest.raises(S.SboError) as e:
        S.Problem.dense(Q, None, precision=S.SBO_FP32)
    assert e.value.status == S.SBO_ERANGE


@pytest.mark.parametrize("second, ok", [(2**23, False), (2**23 - 1, True)])
def test_row_sums_span_tiles(second, ok):
    """Row 5's |A| sum is gathered from two tiles above the diagonal (columns 70 and 150), rows 70
    and 150 from tiles below it: 2^23 + 2^23 reaches 2^24 and is rejected (A b would not be exact
    in FP32), one less is accepted and evaluates exactly."""
    import oracle.pdbo as O
    build_lib()
    n = 200
    Q = np.zeros((n, n), np.int32)
    Q[5, 70] = 2**23
    Q[150, 5] = second
    if not ok:
        with pytest.raises(S.SboError) as e:
            S.Problem.dense(Q, None, precision=S.SBO_FP32)
        assert e.value.status == S.SBO_ERANGE
        return
    bits = np.zeros((3, n), np.uint8)
    bits[0, [5, 70]] = 1
    bits[1, [5, 150]] = 1
    bits[2, [5, 70, 150]] = 1
    with S.Problem.dense(Q, None, precision=S.SBO_FP32) as P:
        F = P.eval(bits)
    assert F.tolist() == O.objective_batch(Q, np.zeros(n, np.int32), bits).tolist()

