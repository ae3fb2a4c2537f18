"""Pins of the oracle's Algorithm 1 and symmetric variant (Sections 2.1-2.2) and the
error bounds of Section 3 (Theorems 2 and 4, Lemmas dbound and qbound)."""
import numpy as np
import pytest

from oracle.kernel import kernel_dense
from oracle.dense import bistochastic_dense, symmetric_dense, top_eigh, lowrank_bistochastic_dense
from oracle.pchol import greedy_pchol, arpc
from oracle.alg1 import bistochastic_evd, symmetric_evd, degree_vectors, NotPositive, constant_eigvec_fix
from oracle import bounds


def _pts(n, d, seed=0):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, d))


def _max_angle(U, V):
    """Largest principal angle (sin) between the column spaces of U and V."""
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    return float(np.linalg.norm(Qv - Qu @ (Qu.T @ Qv), 2))


def test_rank_one_closed_form():
    # F = c 1/sqrt(N): P~ = 1 1^T / N, one eigenvalue 1 with eigenvector 1/sqrt(N)
    N = 9
    F = np.full((N, 1), 0.7 / np.sqrt(N))
    lam, U = bistochastic_evd(F)
    assert abs(lam[0] - 1.0) < 1e-14
    assert np.allclose(np.abs(U[:, 0]), 1 / np.sqrt(N), atol=1e-14)
    d, q = degree_vectors(F)
    assert np.allclose(d, 0.49) and np.allclose(q, 1.0)


def test_two_cluster_closed_form():
    # block-diagonal K~: two eigenvalues 1 with cluster-indicator eigenvectors
    F = np.zeros((5, 2))
    F[:2, 0] = 0.8
    F[2:, 1] = 1.3
    lam, U = bistochastic_evd(F)
    assert np.allclose(lam, [1.0, 1.0], atol=1e-14)
    ind = np.zeros((5, 2))
    ind[:2, 0] = 1
    ind[2:, 1] = 1
    assert _max_angle(U, ind) < 1e-12


def test_alg1_equals_dense_lowrank_P():
    X = _pts(150, 3, 1)
    eps = 4.0
    F, S, _, _ = greedy_pchol(X, eps, 30)
    lam, U = bistochastic_evd(F, k=12)
    Pt, _, _ = lowrank_bistochastic_dense(F)
    lam_d, U_d = top_eigh(Pt, 12)
    assert np.max(np.abs(lam - lam_d) / np.abs(lam_d)) < 1e-10
    # compare eigenvectors through P~ itself: P~ U = U Lambda and orthonormality
    assert np.max(np.abs(Pt @ U - U * lam)) < 1e-12
    assert np.max(np.abs(U.T @ U - np.eye(12))) < 1e-12
    # unit row sums: 1 is an eigenvalue of P~ with eigenvector 1/sqrt(N)
    assert np.allclose(Pt.sum(1), 1.0, atol=1e-12)
    i1 = int(np.argmin(np.abs(lam - 1.0)))
    assert abs(lam[i1] - 1.0) < 1e-12
    assert np.allclose(np.abs(U[:, i1]), 1 / np.sqrt(150), atol=1e-10)


def test_full_rank_equals_dense_P():
    X = _pts(80, 2, 2)
    eps = 0.2
    K = kernel_dense(X, eps)
    F, S, _, _ = greedy_pchol(X, eps, 80)
    lam, U = bistochastic_evd(F, k=10)
    P, _, _ = bistochastic_dense(K)
    lam_d, U_d = top_eigh(P, 10)
    assert np.max(np.abs(lam - lam_d)) < 1e-10
    assert np.max(np.abs(P @ U - U * lam)) < 1e-9


def test_symmetric_variant_equals_dense():
    X = _pts(100, 3, 3)
    F, _, _, _ = greedy_pchol(X, 3.0, 25)
    lam, U = symmetric_evd(F, k=8)
    Lt, _ = symmetric_dense(F @ F.T)
    lam_d, _ = top_eigh(Lt, 8)
    assert np.max(np.abs(lam - lam_d)) < 1e-12
    assert np.max(np.abs(Lt @ U - U * lam)) < 1e-12
    # SVD form (C = I): eigenvalues are the squared singular values of D~^-1/2 F
    d = F @ (F.T @ np.ones(100))
    sv = np.linalg.svd(F / np.sqrt(d)[:, None], compute_uv=False)
    assert np.allclose(lam, sv[:8] ** 2, atol=1e-13)


def test_positivity_asserts():
    F = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])   # row sums of F F^T: 0 for rows 0 and 2
    with pytest.raises(NotPositive):
        degree_vectors(F)


def test_constant_eigvec_fix():
    U = np.linalg.qr(_pts(20, 4, 4))[0]
    V = constant_eigvec_fix(U)
    assert np.allclose(np.abs(V[:, 0]), 1 / np.sqrt(20))
    assert np.max(np.abs(V.T @ V - np.eye(4))) < 1e-13


@pytest.mark.parametrize("r", [10, 25, 60])
def test_error_bounds_hold(r):
    X = _pts(120, 2, 5)
    eps = 1.5
    K = kernel_dense(X, eps)
    out = arpc(X, eps, r, 5, seed=r)
    Kt = out["F"] @ out["F"].T
    a, b, c, e = bounds.lemma_dbound(K, Kt)
    assert a <= b and c <= e
    a, b = bounds.lemma_qbound(K, Kt)
    assert a <= b
    a, b = bounds.theorem4_bound(K, Kt)
    assert a <= b
    a, b = bounds.theorem2_bound(K, Kt)
    assert a <= b


def test_trace_norm_error_decreases_with_rank():
    X = _pts(200, 3, 6)
    errs = [200 - np.sum(arpc(X, 2.0, r, 8, seed=1)["F"] ** 2) for r in (8, 32, 96)]
    assert errs[0] > errs[1] > errs[2] >= 0
