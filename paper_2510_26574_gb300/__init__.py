"""GB300-native low-rank eigendecomposition of bistochastic kernel matrices.

Implements the method of Vales & Giannakis, "Accelerated decomposition of
bistochastic kernel matrices by low rank approximation" (arXiv 2510.26574):
pivoted partial Cholesky of an implicit Gaussian kernel matrix (greedy or
accelerated randomly pivoted Cholesky), bistochastic normalisation from the
factor, and the top-k eigenpairs, in hand-written sm_103a CUDA kernels behind
the C-ABI of include/kevd.h (libkevd.so), with the thin binding in kevd.py.
"""
from .kevd import (rpchol_factor, bistoch_normalize, eig_topk, workspace_bytes, status_string, KevdError,
                   lib, LIB_PATH, EXPORTS, STAGES, trace_enable, trace_reset, trace_read, Batch,
                   symmetric_normalize, symmetric_eig_topk, constant_eigvec_fix, rpchol_factor_lowmem,
                   bistoch_normalize_lowmem, eig_topk_lowmem, kernel_exp)

__all__ = ["rpchol_factor", "bistoch_normalize", "eig_topk", "workspace_bytes", "status_string", "KevdError",
           "lib", "LIB_PATH", "EXPORTS", "STAGES", "trace_enable", "trace_reset", "trace_read", "Batch",
           "symmetric_normalize", "symmetric_eig_topk", "constant_eigvec_fix", "rpchol_factor_lowmem",
           "bistoch_normalize_lowmem", "eig_topk_lowmem", "kernel_exp"]
