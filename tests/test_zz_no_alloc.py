"""sbo_lagrangian_noalloc against sbo_lagrangian, through the C ABI.

The allocation-free entry point exists for callers that may not call cudaMalloc (code inside a
CUDA stream capture, processes whose device memory belongs to a framework's pool or a fixed
budget, loops that cannot absorb an allocation's implicit synchronisation).  It must give the
same values and gradients as the allocating entry point, call after call, even though every call
reuses the same fixed scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

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
