"""Delay embeddings of KS grid data into point clouds (Section 4, delay map W)."""
import numpy as np


def delay_embed_vsa(u, J):
    """Points (t, x_m) -> (u(t, x_m), u(t-1, x_m), ..., u(t-J+1, x_m)).

    ``u`` has shape (T, M).  Returns X of shape ((T-J+1)*M, J), rows ordered
    time-major (row = t*M + m), the product-space sampling of the vector-valued
    spectral analysis map with J delays at one grid point.
    """
    T, M = u.shape
    nt = T - J + 1
    X = np.empty((nt, M, J), dtype=u.dtype)
    for lag in range(J):
        X[:, :, lag] = u[J - 1 - lag: J - 1 - lag + nt, :]
    return X.reshape(nt * M, J)


def delay_embed_neighbours(u, q):
    """Points (t, x_m) -> q delays at x_{m-1}, x_m, x_{m+1} (periodic), concatenated.

    Returns X of shape ((T-q+1)*M, 3q), rows ordered time-major.
    """
    T, M = u.shape
    nt = T - q + 1
    blocks = []
    for shift in (1, 0, -1):                         # x_{m-1}, x_m, x_{m+1}
        us = np.roll(u, shift, axis=1)
        blocks.append(delay_embed_vsa(us, q).reshape(nt, M, q))
    return np.concatenate(blocks, axis=2).reshape(nt * M, 3 * q)
