"""Pins of the oracle's kernel and dense normalised matrices (Section 1.1)."""
import math

import numpy as np

from oracle.kernel import kernel_block, kernel_dense
from oracle.dense import bistochastic_dense, symmetric_dense, top_eigh


def _pts(n, d, seed=0):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, d))


def test_kernel_hand_value():
    # |(0,0)-(3,4)|^2 = 25, eps = 25 -> exp(-1)
    assert kernel_block([[0.0, 0.0]], [[3.0, 4.0]], 25.0)[0, 0] == math.exp(-1.0)


def test_kernel_brute_force_and_asm1():
    X = _pts(7, 3)
    eps = 2.5
    K = kernel_dense(X, eps)
    for i in range(7):
        for j in range(7):
            s = sum((X[i][c] - X[j][c]) ** 2 for c in range(3))
            assert abs(K[i, j] - math.exp(-s / eps)) < 1e-15
    # Assumption 1: positive, symmetric, PSD, k(x,x)=1
    assert np.all(K > 0)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.0)
    assert np.linalg.eigvalsh(K).min() > -1e-12


def test_bistochastic_brute_force():
    X = _pts(6, 2, 1)
    K = kernel_dense(X, 1.3)
    P, d, q = bistochastic_dense(K)
    N = 6
    dd = [sum(K[i]) for i in range(N)]
    qq = [sum(K[i][w] / dd[w] for w in range(N)) for i in range(N)]
    for i in range(N):
        for j in range(N):
            pij = sum(K[i][w] * K[w][j] / (dd[i] * qq[w] * dd[j]) for w in range(N))
            assert abs(P[i, j] - pij) < 1e-14
    assert np.allclose(d, dd, rtol=0, atol=1e-14) and np.allclose(q, qq, rtol=0, atol=1e-14)


def test_bistochastic_markov_properties():
    X = _pts(120, 4, 2)
    K = kernel_dense(X, 3.0)
    P, _, _ = bistochastic_dense(K)
    assert np.allclose(P.sum(1), 1.0, atol=1e-13)
    assert np.allclose(P, P.T, atol=1e-15)
    assert np.all(P > 0)
    lam, U = top_eigh(P, 120)
    assert abs(lam[0] - 1.0) < 1e-12
    assert lam.min() > -1e-12 and lam.max() < 1 + 1e-12
    u0 = U[:, 0] * np.sign(U[0, 0])
    assert np.allclose(u0, 1 / np.sqrt(120), atol=1e-10)


def test_symmetric_brute_force():
    X = _pts(5, 2, 3)
    K = kernel_dense(X, 0.7)
    L, d = symmetric_dense(K)
    for i in range(5):
        for j in range(5):
            assert abs(L[i, j] - K[i, j] / math.sqrt(sum(K[i]) * sum(K[j]))) < 1e-15
