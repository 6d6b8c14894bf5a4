"""ctypes binding of libsbo (include/sbo.h): same names, argument marshalling only.

Every function here converts Python/numpy/torch arguments to the C types of the entry point
with the same name and raises :class:`SboError` on a non-OK status.  No step of the method runs
in Python.  The library is loaded from this package's ``_lib/libsbo.so``; importing a function
that needs it raises when the library has not been built (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsbo.so")

SBO_OK, SBO_EINVAL, SBO_ENOMEM, SBO_ECUDA, SBO_ETIMEOUT, SBO_ENOTREADY, SBO_ERANGE, SBO_EDEVICE = range(8)
STATUS_NAMES = ["SBO_OK", "SBO_EINVAL", "SBO_ENOMEM", "SBO_ECUDA", "SBO_ETIMEOUT", "SBO_ENOTREADY",
                "SBO_ERANGE", "SBO_EDEVICE"]
SBO_FP32, SBO_BF16, SBO_FP8_E4M3 = 0, 1, 2
SBO_OPT_KERNEL, SBO_OPT_USE_GRAPH, SBO_OPT_TILE_N, SBO_OPT_TIMEOUT_US, SBO_OPT_SPLIT_K, SBO_OPT_AUTOTUNE, \
    SBO_OPT_PDL, SBO_OPT_DUAL, SBO_OPT_G, SBO_OPT_KEEP_GRAD, SBO_OPT_CSR_FORM, SBO_OPT_EVAL_MODE, \
    SBO_OPT_STEPS_PER_LAUNCH = 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13
EVAL_MODE_RULE, EVAL_MODE_INLINE, EVAL_MODE_BESIDE = 0, 1, 2
CSR_FORM_AUTO, CSR_FORM_ROW1, CSR_FORM_ROW2, CSR_FORM_PIPE2, CSR_FORM_STAGED = 0, 1, 2, 3, 4
CSR_FORM_ROW1_STREAM, CSR_FORM_ROW2_STREAM, CSR_FORM_PIPE2_STREAM, CSR_FORM_RESIDENT = 5, 6, 7, 8
G_QUADRATIC, G_ENTROPY = 0, 1
DUAL_COORDINATE, DUAL_SINGLE = 0, 1
KERNEL_AUTO, KERNEL_SIMT, KERNEL_TC, KERNEL_TINY, KERNEL_CSR, KERNEL_MAXK = 0, 1, 2, 3, 4, 5

# every symbol include/sbo.h declares
EXPORTS = ["sbo_create_dense", "sbo_create_dense_i8", "sbo_create_csr", "sbo_create_maxkcut",
           "sbo_gda_start", "sbo_gda_start_xy", "sbo_gda_run", "sbo_gda", "sbo_sync",
           "sbo_eval", "sbo_best", "sbo_restart_best", "sbo_state", "sbo_gradient", "sbo_trace",
           "sbo_lagrangian", "sbo_lagrangian_noalloc", "sbo_dual_bound",
           "sbo_set_option", "sbo_info", "sbo_launch_count", "sbo_destroy", "sbo_last_error", "sbo_version",
           "sbo_group_create", "sbo_group_start", "sbo_group_run", "sbo_group_sync", "sbo_group_set_option",
           "sbo_group_launch_count", "sbo_group_destroy"]


class SboError(RuntimeError):
    def __init__(self, status: int, message: str, call: str):
        self.status = status
        self.message = message
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{call}: {name}: {message}")


class sbo_gda_params(ctypes.Structure):
    _fields_ = [("restarts", ctypes.c_int32), ("eval_every", ctypes.c_int32), ("iters", ctypes.c_int64),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double), ("ybar", ctypes.c_double),
                ("delta", ctypes.c_double), ("grad_tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


_lib = None
_P = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_U8P = ctypes.POINTER(ctypes.c_uint8)
_F32P = ctypes.POINTER(ctypes.c_float)


def lib():
    """The loaded libsbo (raises FileNotFoundError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(f"{LIB_PATH} is missing: build it with "
                                "`python -m paper_2509_21064_gb300.build` (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    sig = {
        "sbo_create_dense": (st, [ctypes.c_int64, _I32P, _I32P, ctypes.c_int32, _P, ctypes.POINTER(_P)]),
        "sbo_create_csr": (st, [ctypes.c_int64, ctypes.c_int64, _I64P, _I32P, _I32P, _I32P, ctypes.c_int32, _P,
                                ctypes.POINTER(_P)]),
        "sbo_create_dense_i8": (st, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int8), _I32P, ctypes.c_int32, _P,
                                     ctypes.POINTER(_P)]),
        "sbo_create_maxkcut": (st, [ctypes.c_int64, ctypes.c_int64, _I32P, _I32P, _I32P, ctypes.c_int32, _P,
                                    ctypes.POINTER(_P)]),
        "sbo_gda_start": (st, [_P, ctypes.POINTER(sbo_gda_params), _F32P]),
        "sbo_dual_bound": (st, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "sbo_gda_start_xy": (st, [_P, ctypes.POINTER(sbo_gda_params), _F32P, _F32P]),
        "sbo_gda_run": (st, [_P, ctypes.c_int64]),
        "sbo_gda": (st, [_P, ctypes.POINTER(sbo_gda_params)]),
        "sbo_sync": (st, [_P]),
        "sbo_eval": (st, [_P, ctypes.c_int64, _U8P, _I64P]),
        "sbo_best": (st, [_P, _U8P, _I64P, _I64P, _I32P]),
        "sbo_restart_best": (st, [_P, _I64P, _I64P]),
        "sbo_state": (st, [_P, _F32P, _F32P]),
        "sbo_gradient": (st, [_P, _F32P]),
        "sbo_trace": (st, [_P, _I64P, ctypes.c_int64, _I64P]),
        "sbo_lagrangian": (st, [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P]),
        "sbo_lagrangian_noalloc": (st, [_P, ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P]),
        "sbo_set_option": (st, [_P, ctypes.c_int32, ctypes.c_int64]),
        "sbo_info": (st, [_P, _I64P, _I32P, _I32P, _I32P, _I64P]),
        "sbo_launch_count": (ctypes.c_int64, [_P]),
        "sbo_destroy": (None, [_P]),
        "sbo_last_error": (ctypes.c_char_p, []),
        "sbo_group_create": (st, [ctypes.c_int32, ctypes.POINTER(_P), _P, ctypes.POINTER(_P)]),
        "sbo_group_start": (st, [_P, ctypes.POINTER(sbo_gda_params)]),
        "sbo_group_run": (st, [_P, ctypes.c_int64]),
        "sbo_group_sync": (st, [_P]),
        "sbo_group_set_option": (st, [_P, ctypes.c_int32, ctypes.c_int64]),
        "sbo_group_launch_count": (ctypes.c_int64, [_P]),
        "sbo_group_destroy": (None, [_P]),
        "sbo_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, call: str):
    if status != SBO_OK:
        raise SboError(status, lib().sbo_last_error().decode(), call)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)       # torch.cuda.Stream


def params(restarts, iters, alpha, beta, ybar, delta=0.01, grad_tol=None, eval_every=10, seed=0, **_):
    """sbo_gda_params from keyword values (grad_tol defaults to 2*delta, as in Algorithm 1)."""
    return sbo_gda_params(int(restarts), int(eval_every), int(iters), float(alpha), float(beta), float(ybar),
                          float(delta), float(2 * delta if grad_tol is None else grad_tol), int(seed) & (2**64 - 1))


# ---- entry points ------------------------------------------------------------------------------
def sbo_create_dense(Q, c=None, precision=SBO_BF16, stream=None):
    """Q as int32; an int8 array goes to sbo_create_dense_i8 (a quarter of the bytes to copy)."""
    Q = np.asarray(Q)
    n = Q.shape[0]
    if Q.ndim != 2 or Q.shape[1] != n:
        raise ValueError("Q must be square")
    cc = None if c is None else np.ascontiguousarray(c, dtype=np.int32)
    h = _P()
    if Q.dtype == np.int8:
        Q = np.ascontiguousarray(Q)
        _check(lib().sbo_create_dense_i8(n, _ptr(Q, ctypes.c_int8), None if cc is None else _ptr(cc, ctypes.c_int32),
                                         int(precision), _stream(stream), ctypes.byref(h)), "sbo_create_dense_i8")
        return h
    Q = np.ascontiguousarray(Q, dtype=np.int32)
    _check(lib().sbo_create_dense(n, _ptr(Q, ctypes.c_int32), None if cc is None else _ptr(cc, ctypes.c_int32),
                                  int(precision), _stream(stream), ctypes.byref(h)), "sbo_create_dense")
    return h


def sbo_create_csr(n, rowptr, col, val, c=None, precision=SBO_FP32, stream=None):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.int32)
    cc = None if c is None else np.ascontiguousarray(c, dtype=np.int32)
    h = _P()
    _check(lib().sbo_create_csr(int(n), int(col.size), _ptr(rowptr, ctypes.c_int64), _ptr(col, ctypes.c_int32),
                                _ptr(val, ctypes.c_int32), None if cc is None else _ptr(cc, ctypes.c_int32),
                                int(precision), _stream(stream), ctypes.byref(h)), "sbo_create_csr")
    return h


def sbo_gda_start(h, prm: sbo_gda_params, x0=None):
    x = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float32)
    _check(lib().sbo_gda_start(h, ctypes.byref(prm), None if x is None else _ptr(x, ctypes.c_float)),
           "sbo_gda_start")


def sbo_gda_start_xy(h, prm: sbo_gda_params, x0=None, y0=None):
    x = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float32)
    y = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float32)
    _check(lib().sbo_gda_start_xy(h, ctypes.byref(prm), None if x is None else _ptr(x, ctypes.c_float),
                                  None if y is None else _ptr(y, ctypes.c_float)), "sbo_gda_start_xy")


def sbo_gda_run(h, iters):
    _check(lib().sbo_gda_run(h, int(iters)), "sbo_gda_run")


def sbo_gda(h, prm: sbo_gda_params):
    _check(lib().sbo_gda(h, ctypes.byref(prm)), "sbo_gda")


def sbo_sync(h):
    _check(lib().sbo_sync(h), "sbo_sync")


def sbo_eval(h, bits):
    b = np.ascontiguousarray(np.atleast_2d(bits), dtype=np.uint8)
    F = np.zeros(b.shape[0], dtype=np.int64)
    _check(lib().sbo_eval(h, b.shape[0], _ptr(b, ctypes.c_uint8), _ptr(F, ctypes.c_int64)), "sbo_eval")
    return F


def sbo_best(h, n):
    x = np.zeros(n, dtype=np.uint8)
    F, t, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().sbo_best(h, _ptr(x, ctypes.c_uint8), ctypes.byref(F), ctypes.byref(t), ctypes.byref(r)),
           "sbo_best")
    return x, F.value, t.value, r.value


def sbo_restart_best(h, B):
    F = np.zeros(B, dtype=np.int64)
    t = np.zeros(B, dtype=np.int64)
    _check(lib().sbo_restart_best(h, _ptr(F, ctypes.c_int64), _ptr(t, ctypes.c_int64)), "sbo_restart_best")
    return F, t


def sbo_create_maxkcut(n, ei, ej, w, k, stream=None):
    ei = np.ascontiguousarray(ei, dtype=np.int32)
    ej = np.ascontiguousarray(ej, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    if not (ei.size == ej.size == w.size):
        raise ValueError("ei, ej and w must have the same length")
    h = _P()
    _check(lib().sbo_create_maxkcut(int(n), int(ei.size), _ptr(ei, ctypes.c_int32), _ptr(ej, ctypes.c_int32),
                                    _ptr(w, ctypes.c_int32), int(k), _stream(stream), ctypes.byref(h)),
           "sbo_create_maxkcut")
    return h


def sbo_dual_bound(h, ybar, alpha, iters):
    """(certified lower bound on min F, L at the final point); see include/sbo.h."""
    lb, val = ctypes.c_double(), ctypes.c_double()
    _check(lib().sbo_dual_bound(h, float(ybar), float(alpha), int(iters), ctypes.byref(lb), ctypes.byref(val)),
           "sbo_dual_bound")
    return lb.value, val.value


def sbo_state(h, B, n, k=1):
    """x (B x n, or B x n x k for Max-k-Cut) and y (B x n)."""
    X = np.zeros((B, n) if k == 1 else (B, n, k), dtype=np.float32)
    Y = np.zeros((B, n), dtype=np.float32)
    _check(lib().sbo_state(h, _ptr(X, ctypes.c_float), _ptr(Y, ctypes.c_float)), "sbo_state")
    return X, Y


def sbo_gradient(h, B, n):
    """dL/dx (B x n) that the latest iteration used (runs started with SBO_OPT_KEEP_GRAD = 1)."""
    G = np.zeros((B, n), dtype=np.float32)
    _check(lib().sbo_gradient(h, _ptr(G, ctypes.c_float)), "sbo_gradient")
    return G


def sbo_trace(h, cap=1 << 16):
    out = np.zeros(cap, dtype=np.int64)
    cnt = ctypes.c_int64()
    _check(lib().sbo_trace(h, _ptr(out, ctypes.c_int64), cap, ctypes.byref(cnt)), "sbo_trace")
    return out[:min(cnt.value, cap)]


def sbo_lagrangian(h, B, X_ptr, Y_ptr, gout_ptr=None, L_ptr=None, GX_ptr=None, GY_ptr=None, stream=None):
    """Device-pointer call (ints from ``tensor.data_ptr()``)."""
    _check(lib().sbo_lagrangian(h, int(B), X_ptr, Y_ptr, gout_ptr, L_ptr, GX_ptr, GY_ptr, _stream(stream)),
           "sbo_lagrangian")


def sbo_lagrangian_noalloc(h, B, X_ptr, Y_ptr, gout_ptr=None, L_ptr=None, GX_ptr=None, GY_ptr=None, stream=None):
    """As sbo_lagrangian, without any device allocation (fixed 16 MiB scratch; see sbo.h)."""
    _check(lib().sbo_lagrangian_noalloc(h, int(B), X_ptr, Y_ptr, gout_ptr, L_ptr, GX_ptr, GY_ptr,
                                        _stream(stream)), "sbo_lagrangian_noalloc")


def sbo_set_option(h, option, value):
    _check(lib().sbo_set_option(h, int(option), int(value)), "sbo_set_option")


def sbo_info(h):
    n, B, k, tn, t = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().sbo_info(h, ctypes.byref(n), ctypes.byref(B), ctypes.byref(k), ctypes.byref(tn), ctypes.byref(t)),
           "sbo_info")
    return {"n": n.value, "restarts": B.value, "kernel": k.value, "tile_n": tn.value, "t": t.value}


def sbo_launch_count(h) -> int:
    return int(lib().sbo_launch_count(h))


def sbo_destroy(h):
    if h:
        lib().sbo_destroy(h)


def sbo_version() -> str:
    return lib().sbo_version().decode()


# ---- a thin owner of a handle ------------------------------------------------------------------
class Problem:
    """Owns one problem handle; every method forwards to the entry point of the same name."""

    def __init__(self, handle, n: int, k: int = 1):
        self.h = handle
        self.n = int(n)
        self.k = int(k)          # parts per vertex (Max-k-Cut), 1 otherwise
        self.restarts = 0

    @classmethod
    def dense(cls, Q, c=None, precision=SBO_BF16, stream=None):
        return cls(sbo_create_dense(Q, c, precision, stream), np.asarray(Q).shape[0])

    @classmethod
    def csr(cls, n, rowptr, col, val, c=None, precision=SBO_FP32, stream=None):
        return cls(sbo_create_csr(n, rowptr, col, val, c, precision, stream), n)

    @classmethod
    def maxkcut(cls, n, ei, ej, w, k, stream=None):
        return cls(sbo_create_maxkcut(n, ei, ej, w, k, stream), n, k)

    def set_option(self, option, value):
        sbo_set_option(self.h, option, value)

    def start(self, prm: sbo_gda_params, x0=None, y0=None):
        if y0 is None:
            sbo_gda_start(self.h, prm, x0)
        else:
            sbo_gda_start_xy(self.h, prm, x0, y0)
        self.restarts = prm.restarts

    def run(self, iters):
        sbo_gda_run(self.h, iters)

    def gda(self, prm: sbo_gda_params):
        sbo_gda(self.h, prm)
        self.restarts = prm.restarts

    def sync(self):
        sbo_sync(self.h)

    def eval(self, bits):
        return sbo_eval(self.h, bits)

    def best(self):
        return sbo_best(self.h, self.n)

    def restart_best(self):
        return sbo_restart_best(self.h, self.restarts)

    def state(self):
        return sbo_state(self.h, self.restarts, self.n, self.k)

    def gradient(self):
        return sbo_gradient(self.h, self.restarts, self.n)

    def dual_bound(self, ybar, alpha, iters):
        self.restarts = 1
        return sbo_dual_bound(self.h, ybar, alpha, iters)

    def trace(self, cap=1 << 16):
        return sbo_trace(self.h, cap)

    def info(self):
        return sbo_info(self.h)

    def launch_count(self):
        return sbo_launch_count(self.h)

    def close(self):
        if self.h:
            sbo_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- grouped runs ----------------------------------------------------------------------------
def sbo_group_create(problems, stream=None):
    arr = (_P * len(problems))(*[pr.h if isinstance(pr, Problem) else pr for pr in problems])
    h = _P()
    _check(lib().sbo_group_create(len(problems), arr, _stream(stream), ctypes.byref(h)), "sbo_group_create")
    return h


def sbo_group_start(g, prms):
    arr = (sbo_gda_params * len(prms))(*prms)
    _check(lib().sbo_group_start(g, arr), "sbo_group_start")


def sbo_group_run(g, iters):
    _check(lib().sbo_group_run(g, int(iters)), "sbo_group_run")


def sbo_group_sync(g):
    _check(lib().sbo_group_sync(g), "sbo_group_sync")


def sbo_group_set_option(g, option, value):
    _check(lib().sbo_group_set_option(g, int(option), int(value)), "sbo_group_set_option")


def sbo_group_launch_count(g) -> int:
    return int(lib().sbo_group_launch_count(g))


def sbo_group_destroy(g):
    if g:
        lib().sbo_group_destroy(g)


class Group:
    """Owns one group handle over caller-owned :class:`Problem` members."""

    def __init__(self, problems, stream=None):
        self.problems = list(problems)
        self.h = sbo_group_create(self.problems, stream)

    def set_option(self, option, value):
        sbo_group_set_option(self.h, option, value)

    def start(self, prms):
        sbo_group_start(self.h, prms)
        for pr, q in zip(self.problems, prms):
            pr.restarts = q.restarts

    def run(self, iters):
        sbo_group_run(self.h, iters)

    def sync(self):
        sbo_group_sync(self.h)

    def launch_count(self):
        return sbo_group_launch_count(self.h)

    def close(self):
        if self.h:
            sbo_group_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
