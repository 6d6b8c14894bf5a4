"""Seeded synthetic workloads shaped like the PDBO paper's (arXiv 2509.21064) experiments.

This package only draws problem data (Q, c, graphs) and hyper-parameters. It holds none of
the method's arithmetic, so the FP64 oracle (``oracle/``) and the CUDA path
(``paper_2509_21064_gb300``) can both be fed from it without sharing any computation.
"""
from .generators import (  # noqa: F401
    dense_qubo,
    maxcut_er,
    maxcut_torus,
    maxcut_regular,
    mis_regular,
    heterogeneous_qubos,
    heterogeneous_qubo,
    heterogeneous_shapes,
    iter_heterogeneous_qubos,
    csr_from_edges,
    maxcut_qubo,
    spectral_scale,
    csr_spectral_scale,
    dense_from_csr,
    dense_params,
    graph_params,
    GdaParams,
)
