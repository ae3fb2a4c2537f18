"""Algorithm 1 (approximate EVD of the bistochastic kernel matrix from F) and the
symmetric-normalisation variant of Section 2.1, written as the paper states them.

Bistochastic (Section 2.2, Algorithm 1):
  D~ = diag(F F^T 1) > 0,  Q~ = diag(F F^T D~^-1 1) > 0,
  D~^-1 F = Q1 R1 (reduced Householder QR),
  R1 (F^T Q~^-1 F) R1^T = V Lambda V^T,  U = Q1 V,  eigenvalues descending.
Symmetric (Section 2.1): D~^-1/2 F = Q R,  R R^T = V Lambda V^T,  U = Q V.
The optional constant-eigenvector fix of Algorithm 1 is provided separately.
"""
import numpy as np


class NotPositive(ValueError):
    pass


def degree_vectors(F):
    """(d~, q~) = (F (F^T 1), F (F^T d~^-1)), with the positivity checks of Algorithm 1."""
    F = np.asarray(F, dtype=np.float64)
    d = F @ (F.T @ np.ones(F.shape[0]))
    if not np.all(d > 0):
        raise NotPositive("diag(D~) not positive")
    q = F @ (F.T @ (1.0 / d))
    if not np.all(q > 0):
        raise NotPositive("diag(Q~) not positive")
    return d, q


def bistochastic_evd(F, k=None):
    """Top-k eigenpairs (Lambda descending, U N x k) of P~ by Algorithm 1."""
    F = np.asarray(F, dtype=np.float64)
    d, q = degree_vectors(F)
    Q1, R1 = np.linalg.qr(F / d[:, None], mode="reduced")
    C = F.T @ (F / q[:, None])
    lam, V = np.linalg.eigh(R1 @ C @ R1.T)
    order = np.argsort(-lam, kind="stable")
    if k is not None:
        order = order[:k]
    return lam[order], Q1 @ V[:, order]


def constant_eigvec_fix(U):
    """Optional last lines of Algorithm 1: U(:,0) = 1/sqrt(N), then re-orthonormalise by QR."""
    U = np.array(U, dtype=np.float64, copy=True)
    U[:, 0] = 1.0 / np.sqrt(U.shape[0])
    Qf, _ = np.linalg.qr(U, mode="reduced")
    return Qf


def symmetric_evd(F, k=None):
    """Top-k eigenpairs of L~ = (D~^-1/2 F)(D~^-1/2 F)^T via QR and the r x r EVD (Section 2.1)."""
    F = np.asarray(F, dtype=np.float64)
    d = F @ (F.T @ np.ones(F.shape[0]))
    if not np.all(d > 0):
        raise NotPositive("diag(D~) not positive")
    Q, R = np.linalg.qr(F / np.sqrt(d)[:, None], mode="reduced")
    lam, V = np.linalg.eigh(R @ R.T)
    order = np.argsort(-lam, kind="stable")
    if k is not None:
        order = order[:k]
    return lam[order], Q @ V[:, order]
