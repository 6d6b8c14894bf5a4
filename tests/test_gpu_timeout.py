"""Failure detection on the GPU without a fault: every device-side wait of the tcgen05 kernel is
bounded; with a budget far shorter than the work, the waits give up, the kernel drains its own
copies and MMAs, frees its tensor memory and returns, and the host reads SBO_ETIMEOUT.  The
context stays usable: the same handle then runs normally and matches a fresh handle exactly."""
import numpy as np
import pytest

import workloads as W
from paper_2509_21064_gb300 import sbo as S
from paper_2509_21064_gb300.build import build as build_lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,B,tile", [(8192, 1024, 128), (4096, 256, 1256), (4096, 256, 2256)])
def test_bounded_waits_report_timeout_and_the_context_survives(n, B, tile):
    """tile 128: persistent single-CTA tiles; 1256, 2256: K split over thread-block clusters (of
    CTA pairs), whose CTAs still reach every cluster barrier after giving up."""
    build_lib()
    Q, c = W.dense_qubo(n, seed=4)
    p = W.dense_params(Q, restarts=B, iters=100, eval_every=10, seed=2)
    prm = S.params(**p.asdict())
    with S.Problem.dense(Q, c, precision=S.SBO_BF16) as P:
        P.set_option(S.SBO_OPT_TILE_N, tile)
        P.set_option(S.SBO_OPT_TIMEOUT_US, 1)          # 1 us: far below one launch
        P.start(prm)
        P.run(3)
        with pytest.raises(S.SboError) as e:
            P.sync()
        assert e.value.status == S.SBO_ETIMEOUT
        P.sync()                                        # the error word was cleared
        P.set_option(S.SBO_OPT_TIMEOUT_US, 4_000_000)
        P.start(prm)
        P.run(20)
        X, Y = P.state()
        assert P.info()["tile_n"] == tile
    with S.Problem.dense(Q, c, precision=S.SBO_BF16) as P2:
        P2.set_option(S.SBO_OPT_TILE_N, tile)
        P2.start(prm)
        P2.run(20)
        X2, Y2 = P2.state()
    assert np.array_equal(X, X2) and np.array_equal(Y, Y2)


def test_resident_sparse_form_times_out_and_recovers():
    """The resident sparse form (grid barrier between the iterations of a launch) with a 1 us
    budget on its only wait, the grid barrier: the launch either gives up (the host then reads
    SBO_ETIMEOUT) or every CTA arrived in time; either way it returns, and the handle then runs
    normally and matches another form bit for bit."""
    build_lib()
    n = 2000
    i, j, w = W.maxcut_er(n, 6.0, seed=1)
    rowptr, col, val, c = W.maxcut_qubo(n, i, j, w)
    prm = S.params(**W.graph_params("maxcut", restarts=256, iters=100, eval_every=10, seed=2).asdict())
    with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P:
        P.set_option(S.SBO_OPT_CSR_FORM, S.CSR_FORM_RESIDENT)
        P.set_option(S.SBO_OPT_TIMEOUT_US, 1)
        P.start(prm)
        P.run(10)
        try:
            P.sync()
        except S.SboError as e:
            assert e.status == S.SBO_ETIMEOUT
        P.set_option(S.SBO_OPT_TIMEOUT_US, 4_000_000)
        P.start(prm)
        P.run(20)
        X, Y = P.state()
    with S.Problem.csr(n, rowptr, col, val, c, precision=S.SBO_FP32) as P2:
        P2.set_option(S.SBO_OPT_CSR_FORM, S.CSR_FORM_ROW1)
        P2.start(prm)
        P2.run(20)
        X2, Y2 = P2.state()
    assert np.array_equal(X, X2) and np.array_equal(Y, Y2)

