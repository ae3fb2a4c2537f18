"""Dense normalised kernel matrices (Section 1.1) and their eigendecompositions.

Bistochastic: D = diag(K 1), Q = diag(K D^-1 1), P = D^-1 K Q^-1 K D^-1.
Symmetric:    L = D^-1/2 K D^-1/2.
These are the exact matrices the low-rank method approximates; they are only
formed for tiny N.
"""
import numpy as np


def bistochastic_dense(K):
    """(P, d, q) for a dense kernel matrix K."""
    K = np.asarray(K, dtype=np.float64)
    one = np.ones(K.shape[0])
    d = K @ one
    q = K @ (one / d)
    P = (K / d[:, None]) @ (K / (q[:, None] * d[None, :]))
    return P, d, q


def symmetric_dense(K):
    """(L, d) for a dense kernel matrix K."""
    K = np.asarray(K, dtype=np.float64)
    d = K @ np.ones(K.shape[0])
    s = 1.0 / np.sqrt(d)
    return s[:, None] * K * s[None, :], d


def top_eigh(M, k):
    """Top-k eigenpairs of a symmetric matrix, eigenvalues descending."""
    lam, V = np.linalg.eigh(np.asarray(M, dtype=np.float64))
    order = np.argsort(-lam, kind="stable")[:k]
    return lam[order], V[:, order]


def lowrank_bistochastic_dense(F):
    """P~ = D~^-1 F F^T Q~^-1 F F^T D~^-1 formed densely from a factor F (tiny N)."""
    F = np.asarray(F, dtype=np.float64)
    Kt = F @ F.T
    return bistochastic_dense(Kt)
