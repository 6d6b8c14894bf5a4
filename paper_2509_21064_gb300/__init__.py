"""GB300 (sm_103a) batched primal-dual GDA for binary optimisation (PDBO, arXiv 2509.21064).

The compute path lives in ``libsbo.so`` (hand-written CUDA, C ABI in ``include/sbo.h``);
:mod:`.sbo` is its ctypes binding and :mod:`.autograd` the ``torch.autograd.Function`` over the
Lagrangian.  Build the library with :func:`build`.
"""
from .build import build  # noqa: F401
from .sbo import (  # noqa: F401
    Problem, Group, SboError, params, sbo_gda_params,
    SBO_FP32, SBO_BF16, SBO_FP8_E4M3,
    SBO_OPT_KERNEL, SBO_OPT_USE_GRAPH, SBO_OPT_TILE_N, SBO_OPT_TIMEOUT_US, SBO_OPT_SPLIT_K, SBO_OPT_AUTOTUNE,
    KERNEL_AUTO, KERNEL_SIMT, KERNEL_TC, KERNEL_TINY, KERNEL_CSR,
)
