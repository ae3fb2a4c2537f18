"""Pins of the low-memory ARPC oracle (F kept as the pivots S and W = F(S,:)).

* Against the pinned ARPC oracle: same proposals, acceptances, pivots, rho and
  rounds; the factor rebuilt row by row as K(i,S) W^-T equals ARPC's F.
* Against the mathematics: W is lower triangular with W W^T = K(S,S) (the
  Cholesky factor of the pivot block, computed densely); at full rank the
  degrees equal those of the dense K and the eigenpairs equal those of the
  dense P = D^-1 K Q^-1 K D^-1 (Section 1.1).
* Against Algorithm 1 at partial rank: degrees, Grams A = F^T D~^-2 F and
  C = F^T Q~^-1 F, and the top-k eigenpairs of P~ (QR route) from ARPC's F.
* Ragged panels (panel sizes that do not divide N) give the same results.
"""
import numpy as np
import pytest

from oracle.kernel import kernel_dense
from oracle.dense import bistochastic_dense, top_eigh
from oracle.pchol import arpc
from oracle.alg1 import bistochastic_evd, degree_vectors
from oracle.lowmem import arpc_lowmem, lowmem_rows, normalize_lowmem, evd_lowmem
from tests.helpers import compare_eigpairs


def _pts(n, d, seed=0):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, d))


CASES = [(400, 3, 2.0, 60, 12, 5), (700, 5, 6.0, 96, 32, 9), (333, 2, 1.0, 50, 7, 3)]


@pytest.mark.parametrize("N,d,eps,r,b,seed", CASES)
def test_same_decisions_as_arpc(N, d, eps, r, b, seed):
    X = _pts(N, d, seed)
    ref = arpc(X, eps, r, b, seed)
    low = arpc_lowmem(X, eps, r, b, seed, panel=97)
    assert low["rounds"] == ref["rounds"]
    assert low["pivots"].tolist() == ref["pivots"].tolist()
    for a, c in zip(low["log"], ref["log"]):
        assert a["proposals"].tolist() == c["proposals"].tolist()
        assert a["accepted"].tolist() == c["accepted"].tolist()
    assert np.max(np.abs(low["rho"] - ref["rho"])) < 1e-12


@pytest.mark.parametrize("N,d,eps,r,b,seed", CASES)
def test_rebuilt_factor_equals_arpc(N, d, eps, r, b, seed):
    X = _pts(N, d, seed)
    ref = arpc(X, eps, r, b, seed)
    low = arpc_lowmem(X, eps, r, b, seed)
    F = lowmem_rows(X, eps, low["pivots"], low["W"], np.arange(N))
    assert F.shape == ref["F"].shape
    assert np.max(np.abs(F - ref["F"])) < 1e-9


@pytest.mark.parametrize("N,d,eps,r,b,seed", CASES)
def test_W_is_cholesky_of_pivot_block(N, d, eps, r, b, seed):
    X = _pts(N, d, seed)
    low = arpc_lowmem(X, eps, r, b, seed)
    S, W = low["pivots"], low["W"]
    KSS = kernel_dense(X[S], eps)
    assert np.max(np.abs(np.triu(W, 1))) == 0.0
    assert np.all(np.diag(W) > 0)
    assert np.max(np.abs(W @ W.T - KSS)) < 1e-12
    assert np.max(np.abs(W - np.linalg.cholesky(KSS))) < 1e-8


def test_full_rank_matches_dense_bistochastic():
    N = 90
    X = _pts(N, 3, 4)
    eps = 0.3                                   # narrow bandwidth: well-conditioned K
    K = kernel_dense(X, eps)
    low = arpc_lowmem(X, eps, N, 1, 0, until_rank=True)
    S, W = low["pivots"], low["W"]
    assert sorted(S.tolist()) == list(range(N))
    F = lowmem_rows(X, eps, S, W, np.arange(N))
    assert np.max(np.abs(F @ F.T - K)) < 1e-10
    P, dd, qd = bistochastic_dense(K)
    dt, qt, A, C = normalize_lowmem(X, eps, S, W, panel=13)
    assert np.max(np.abs(dt - dd) / dd) < 1e-10
    assert np.max(np.abs(qt - qd) / qd) < 1e-10
    lam, U = evd_lowmem(X, eps, S, W, 10, panel=13)
    lam_d, U_d = top_eigh(P, 10)
    assert abs(lam[0] - 1.0) < 1e-10           # P is bistochastic: top eigenvalue 1
    erel, ang = compare_eigpairs(lam_d, U_d, lam, U, lam_full=top_eigh(P, N)[0])
    assert erel < 1e-9 and ang < 1e-7, (erel, ang)


@pytest.mark.parametrize("N,d,eps,r,b,seed", CASES)
def test_normalize_and_evd_match_algorithm1(N, d, eps, r, b, seed):
    X = _pts(N, d, seed)
    F = arpc(X, eps, r, b, seed)["F"]
    low = arpc_lowmem(X, eps, r, b, seed)
    S, W = low["pivots"], low["W"]
    dd, qd = degree_vectors(F)
    dt, qt, A, C = normalize_lowmem(X, eps, S, W, panel=61)
    assert np.max(np.abs(dt - dd) / dd) < 1e-10
    assert np.max(np.abs(qt - qd) / qd) < 1e-10
    A_ref = F.T @ (F / (dd ** 2)[:, None])
    C_ref = F.T @ (F / qd[:, None])
    assert np.max(np.abs(A - A_ref)) < 1e-9 * np.max(np.abs(A_ref))
    assert np.max(np.abs(C - C_ref)) < 1e-9 * np.max(np.abs(C_ref))
    k = 8
    lam_r, U_r = bistochastic_evd(F)
    lam, U = evd_lowmem(X, eps, S, W, k, panel=61)
    assert np.all(np.diff(lam) <= 0)
    erel, ang = compare_eigpairs(lam_r[:k], U_r[:, :k], lam, U, lam_full=lam_r)
    assert erel < 1e-9 and ang < 1e-6, (erel, ang)


def test_panel_size_does_not_change_results():
    N, r, b = 500, 64, 16
    X = _pts(N, 4, 8)
    eps = 3.0
    a = arpc_lowmem(X, eps, r, b, 2, panel=1)
    c = arpc_lowmem(X, eps, r, b, 2, panel=4096)
    assert a["pivots"].tolist() == c["pivots"].tolist()
    assert np.max(np.abs(a["rho"] - c["rho"])) < 1e-13
    d1 = normalize_lowmem(X, eps, a["pivots"], a["W"], panel=37)
    d2 = normalize_lowmem(X, eps, a["pivots"], a["W"], panel=N)
    for u, v in zip(d1, d2):
        assert np.max(np.abs(u - v)) < 1e-12 * max(1.0, np.max(np.abs(v)))


def test_no_array_of_N_by_r_entries():
    """The state kept across rounds is O(N + r^2): rho (N), S (r), W (r x r)."""
    N, r, b = 2000, 40, 8
    X = _pts(N, 2, 1)
    low = arpc_lowmem(X, 2.0, r, b, 0, panel=256)
    k = len(low["pivots"])
    assert low["W"].shape == (k, k)
    assert low["rho"].shape == (N,)
