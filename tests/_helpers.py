"""Shared helpers of the GPU parity tests: trajectories from the CUDA path (through the C ABI)
and from the FP64 oracle on the same seeded inputs, and the normwise error metric."""
import numpy as np

import oracle as O
from paper_2509_21064_gb300 import sbo as S


def normwise(a, b):
    """Per-row ||a - b||_inf / ||b||_inf (rows are restarts; last axis is the coordinate)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    num = np.max(np.abs(a - b), axis=-1)
    den = np.maximum(np.max(np.abs(b), axis=-1), 1e-30)
    return num / den


def gpu_trajectory(prob: S.Problem, prm, steps, x0=None):
    """States (X, Y) at t = 0..steps, stepping one iteration per sbo_gda_run call."""
    prob.start(prm, x0)
    X, Y = prob.state()
    xs, ys = [X], [Y]
    for _ in range(steps):
        prob.run(1)
        X, Y = prob.state()
        xs.append(X)
        ys.append(Y)
    return np.array(xs), np.array(ys)


def oracle_trajectory(Q, c, prm, steps, X0=None, A=None, cp=None, restarts=None):
    """Oracle states at t = 0..steps and gradients d^t for t < steps (restart subset optional)."""
    if A is None:
        A, cp = O.canonicalize(Q, c)
    n = A.shape[0]
    if X0 is None:
        X0, _ = O.init_state(n, prm.restarts, prm.seed, prm.ybar)
    X = np.array(X0, dtype=np.float64)
    if restarts is not None:
        X = X[restarts]
    Y = np.full_like(X, prm.ybar)
    xs, ys, ds = [X], [Y], []
    for _ in range(steps):
        X, Y, D = O.gda_step(A, cp, X, Y, prm.alpha, prm.beta, prm.delta, prm.grad_tol)
        xs.append(X)
        ys.append(Y)
        ds.append(D)
    return np.array(xs), np.array(ys), np.array(ds)


def to_gda_params(p) -> S.sbo_gda_params:
    return S.params(**p.asdict())
