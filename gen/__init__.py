"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package only draws random sparsity patterns, row lengths and dense fills. It holds
none of the SpMM / SDDMM arithmetic, so the oracle and the CUDA path can both take their
inputs from it without sharing any of the method.
"""
from .csr import (  # noqa: F401
    CSR,
    nnz_for,
    csr_from_lengths,
    csr_uniform,
    csr_powerlaw,
    csr_clustered,
    csr_banded,
    csr_blocked,
    csr_from_triplets,
    gnn_graph,
    gnn_batch,
    gnn_alpha,
    dense_normal,
    dense_uniform,
    dense_int,
    vals_int,
)
from .corpus import corpus_matrix, corpus_spec, extrapolation_spec  # noqa: F401
