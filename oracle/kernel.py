"""Gaussian kernel entries (Section 4, Eq. (data-kernel); Assumption 1).

k(x, y) = exp(-|x - y|^2 / eps).  The paper writes the bandwidth as eps*J for J
delays; the caller folds any such factor into eps.  Squared distances are the
sum of squared coordinate differences (the definition, not the norm expansion).
"""
import numpy as np
from scipy.spatial.distance import cdist


def kernel_block(X, Y, eps):
    """K(X, Y)_ij = exp(-|x_i - y_j|^2 / eps), float64."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    return np.exp(-cdist(X, Y, "sqeuclidean") / eps)


def kernel_columns(X, idx, eps):
    """The columns K(:, idx) of the N x N kernel matrix, shape (N, len(idx))."""
    X = np.asarray(X, dtype=np.float64)
    return kernel_block(X, X[np.asarray(idx, dtype=np.int64)], eps)


def kernel_dense(X, eps):
    """The full N x N kernel matrix (tiny N only)."""
    return kernel_block(X, X, eps)
