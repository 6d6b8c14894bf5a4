"""Shared helpers of the GPU parity tests: trajectories from the CUDA path (through the C ABI)
and from the FP64 oracle on the same seeded inputs, the normwise error metric, and the record of
measured errors."""
import json
import os

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


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), as the tensor-core and BF16 sparse paths
    round the contraction operand x from its FP32 master."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gpu_gradient_trajectory(prob: S.Problem, prm, steps, x0=None):
    """States (X, Y) at t = 0..steps and the gradients d^t (t < steps) the update kernel used,
    stepping one iteration per sbo_gda_run call (the run keeps its gradient: SBO_OPT_KEEP_GRAD)."""
    prob.set_option(S.SBO_OPT_KEEP_GRAD, 1)
    prob.start(prm, x0)
    X, Y = prob.state()
    xs, ys, ds = [X], [Y], []
    for _ in range(steps):
        prob.run(1)
        ds.append(prob.gradient())
        X, Y = prob.state()
        xs.append(X)
        ys.append(Y)
    return np.array(xs), np.array(ys), np.array(ds)


def own_point_gradient(A, cp, X, Y, operand_bf16=False):
    """The oracle's dL/dx (section 3.1 Lagrangian, g(x) = x^2 - x) at the GPU's own iterate
    (X, Y); with operand_bf16 the contraction A x takes x rounded to BF16, the operand the BF16
    paths feed their contraction, so only FP32 accumulation separates the two."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Xc = bf16_round(X) if operand_bf16 else X
    return np.asarray((A @ Xc.T).T) + cp[None, :] + Y * O.g_prime(X)


def gradient_scale(A, cp, X, Y, operand_bf16=False):
    """Magnitude of the summands of dL/dx = A x + c' + y g'(x) per coordinate:
    |A| |x| + |c'| + |y g'(x)| (x rounded to BF16 in the contraction when operand_bf16).  The
    gradient is a sum whose terms cancel as the iteration nears a stationary point; rounding
    errors scale with these summands, not with the gradient itself."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Xc = bf16_round(X) if operand_bf16 else X
    absA = abs(A)
    return np.asarray((absA @ np.abs(Xc).T).T) + np.abs(cp)[None, :] + np.abs(Y * O.g_prime(X))


def scaled_error(d, ref, scale):
    """Per row (restart): ||d - ref||_inf / ||scale||_inf, the gradient's error measured against
    the magnitude of its summands (gradient_scale)."""
    d = np.asarray(d, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    num = np.max(np.abs(d - ref), axis=-1)
    den = np.maximum(np.max(np.asarray(scale), axis=-1), 1e-30)
    return num / den


def report(record: str, **values):
    """Append one JSON line of measured errors to the file named by SBO_PARITY_REPORT (if set)."""
    path = os.environ.get("SBO_PARITY_REPORT")
    if not path:
        return
    with open(path, "a") as f:
        f.write(json.dumps({"record": record, **{k: (float(v) if isinstance(v, (np.floating, float)) else v)
                                                 for k, v in values.items()}}) + "\n")
