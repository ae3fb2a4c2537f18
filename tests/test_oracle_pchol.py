"""Pins of the oracle's pivoted partial Cholesky (Section 1.2, Appendix A)."""
import numpy as np
import pytest

from oracle.kernel import kernel_dense
from oracle.pchol import greedy_pchol, arpc, reject, inverse_cdf
from oracle.philox import uniforms


def _pts(n, d, seed=0):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, d))


def _dense_greedy(K, r):
    """Brute force: explicit Schur complement E, pivot = argmax diag(E)."""
    E = np.array(K, dtype=np.float64)
    piv = []
    for _ in range(r):
        s = int(np.argmax(np.diag(E)))
        if E[s, s] <= 0:
            break
        piv.append(s)
        E = E - np.outer(E[:, s], E[s, :]) / E[s, s]
    return piv, E


def test_greedy_full_rank_reproduces_K_and_is_cholesky():
    X = _pts(60, 3, 1)
    eps = 0.3                       # narrow bandwidth: well-conditioned K
    K = kernel_dense(X, eps)
    assert np.linalg.cond(K) < 1e6
    F, S, rho, _ = greedy_pchol(X, eps, 60)
    assert len(S) == 60 and sorted(S.tolist()) == list(range(60))
    assert np.max(np.abs(K - F @ F.T)) < 1e-12
    # F(S,:) is the (unique) Cholesky factor of K(S,S)
    FS = F[S]
    assert np.max(np.abs(np.triu(FS, 1))) < 1e-12      # zero up to rounding
    assert np.max(np.abs(FS - np.linalg.cholesky(K[np.ix_(S, S)]))) < 1e-12


def test_greedy_pivots_match_dense_schur_brute_force():
    X = _pts(200, 4, 2)
    eps = 4.0
    K = kernel_dense(X, eps)
    F, S, rho, hist = greedy_pchol(X, eps, 40)
    piv, E = _dense_greedy(K, 40)
    assert S.tolist() == piv
    assert np.max(np.abs(rho - np.maximum(np.diag(E), 0))) < 1e-12
    assert np.all(np.diff(hist) <= 1e-15)               # trace error never grows


def test_greedy_tie_goes_to_lowest_index():
    X = np.zeros((5, 2))
    X[3] = [10.0, 0.0]
    F, S, rho, _ = greedy_pchol(X, 1.0, 2)
    assert S.tolist() == [0, 3]                          # rho all equal at start -> index 0


def test_inverse_cdf_definition_and_law():
    rho = np.array([0.0, 2.0, 0.0, 1.0, 5.0, 0.0])
    c = np.cumsum(rho)
    u = np.array([0.0, 0.249, 0.25, 0.3749, 0.375, 0.999999])
    j, _ = inverse_cdf(rho, u)
    for uu, jj in zip(u, j):
        assert c[jj] > uu * c[-1] and (jj == 0 or c[jj - 1] <= uu * c[-1])
    assert j.tolist() == [1, 1, 3, 3, 4, 4]
    # chi-square of many draws against rho / sum(rho)
    rho = np.array([1.0, 3.0, 0.5, 0.0, 2.5, 1.0])
    u = uniforms(99, 0, 0, 40000)
    j, _ = inverse_cdf(rho, u)
    cnt = np.bincount(j, minlength=6)
    assert cnt[3] == 0
    p = rho / rho.sum()
    nz = p > 0
    chi2 = np.sum((cnt[nz] - 40000 * p[nz]) ** 2 / (40000 * p[nz]))
    assert chi2 < 20.5                                   # df=4, p ~ 4e-4


def test_reject_factor_is_cholesky_of_accepted_block():
    X = _pts(30, 3, 4)
    K = kernel_dense(X, 2.0)
    prop = np.array([3, 7, 3, 11, 20, 7, 1, 29])         # with duplicates
    H = K[np.ix_(prop, prop)]
    z = uniforms(5, 1, 0, len(prop))
    T, L, _ = reject(H, z)
    assert 3 not in prop[T][1:].tolist() or prop[T].tolist().count(3) == 1
    assert len(set(prop[T].tolist())) == len(T)          # duplicates rejected
    assert np.max(np.abs(L - np.linalg.cholesky(H[np.ix_(T, T)]))) < 1e-13
    # b=1: always accepted
    T1, L1, _ = reject(H[:1, :1], np.array([0.999999]))
    assert T1.tolist() == [0] and abs(L1[0, 0] - 1.0) < 1e-15


def test_reject_acceptance_law():
    # H = [[1, c], [c, 1]]: the second proposal survives with probability 1 - c^2
    c = 0.6
    H = np.array([[1.0, c], [c, 1.0]])
    n = 20000
    acc = 0
    for i in range(n):
        z = uniforms(3, 1, i, 2)
        T, _, _ = reject(H, z)
        acc += int(1 in T.tolist())
    p = 1 - c * c
    assert abs(acc / n - p) < 4 * np.sqrt(p * (1 - p) / n)


def _dense_rpc(K, r, seed):
    """Brute force RPC (b=1): explicit Schur complement, inverse-CDF sampling."""
    E = np.array(K, dtype=np.float64)
    piv = []
    for i in range(r):
        dg = np.maximum(np.diag(E), 0)
        u = uniforms(seed, 0, i, 1)
        s = int(inverse_cdf(dg, u)[0][0])
        piv.append(s)
        E = E - np.outer(E[:, s], E[s, :]) / E[s, s]
    return piv


def test_arpc_block1_is_rpc():
    X = _pts(150, 3, 5)
    eps = 3.0
    K = kernel_dense(X, eps)
    out = arpc(X, eps, 25, 1, seed=11)
    assert out["pivots"].tolist() == _dense_rpc(K, 25, 11)


def test_arpc_invariants():
    X = _pts(300, 4, 6)
    eps = 5.0
    K = kernel_dense(X, eps)
    out = arpc(X, eps, 64, 16, seed=7)
    F, S, rho = out["F"], out["pivots"], out["rho"]
    k = F.shape[1]
    assert 0 < k <= 64 and len(set(S.tolist())) == k
    R = K - F @ F.T
    # residual diagonal and trace error (Appendix A)
    assert np.max(np.abs(rho - np.maximum(np.diag(R), 0))) < 1e-12
    assert abs(rho.sum() - (300 - np.sum(F * F))) < 1e-10
    # Assumption 2: K >= F F^T >= 0
    assert np.linalg.eigvalsh(R).min() > -1e-10
    # Nystrom identity: F F^T = K(:,S) K(S,S)^+ K(S,:)
    Kn = K[:, S] @ np.linalg.pinv(K[np.ix_(S, S)], rcond=1e-13) @ K[S, :]
    assert np.max(np.abs(Kn - F @ F.T)) < 1e-8
    # F(S,:) lower triangular in acceptance order
    assert np.max(np.abs(np.triu(F[S], 1))) < 1e-10
    sums = [lg["sum_rho"] for lg in out["log"]]
    assert all(b <= a + 1e-12 for a, b in zip(sums, sums[1:]))


def test_arpc_until_rank_exact():
    X = _pts(400, 3, 8)
    out = arpc(X, 2.0, 96, 32, seed=3, until_rank=True)
    assert out["F"].shape[1] == 96
    out2 = arpc(X, 2.0, 96, 32, seed=3)
    assert out2["F"].shape[1] <= 96 and out2["rounds"] == 3


def test_arpc_is_deterministic_per_seed():
    X = _pts(200, 3, 9)
    a = arpc(X, 2.0, 40, 8, seed=5)
    b = arpc(X, 2.0, 40, 8, seed=5)
    c = arpc(X, 2.0, 40, 8, seed=6)
    assert np.array_equal(a["F"], b["F"]) and a["pivots"].tolist() == b["pivots"].tolist()
    assert a["pivots"].tolist() != c["pivots"].tolist()


def test_theorem1_expectation_bound():
    """Theorem 1: E tr(K - K~) <= (1+eps) tr(K - [K]_r') once r is large enough."""
    from oracle.bounds import theorem1_rank, best_rank_error
    X = _pts(120, 2, 10)
    eps = 1.0
    K = kernel_dense(X, eps)
    rp, e = 4, 1.0
    best = best_rank_error(K, rp)
    eta = best / np.trace(K)
    r = int(np.ceil(theorem1_rank(rp, e, eta)))
    assert r < 120
    errs = [120 - np.sum(arpc(X, eps, r, 1, seed=s)["F"] ** 2) for s in range(200)]
    assert np.mean(errs) <= (1 + e) * best


# --------------------------------------------------------------------------
# Replay: the factor of a given pivot sequence
# --------------------------------------------------------------------------
def test_replay_of_arpc_pivots_equals_arpc():
    """Fed ARPC's own accepted pivots (with its per-round block lengths, or one
    pivot per block), the replay reproduces ARPC's F and rho."""
    from oracle.pchol import pchol_given_pivots
    X = _pts(400, 4, 11)
    eps = 6.0
    ref = arpc(X, eps, 96, 16, 42)
    blocks = [len(lg["accepted"]) for lg in ref["log"] if len(lg["accepted"])]
    for bl in (blocks, None):
        rp = pchol_given_pivots(X, eps, ref["pivots"], blocks=bl)
        assert np.max(np.abs(rp["F"] - ref["F"])) < 1e-12
        assert np.max(np.abs(rp["rho"] - ref["rho"])) < 1e-12


def test_replay_is_nystrom_and_cholesky_of_pivot_block():
    """F F^T = K(:,S) K(S,S)^-1 K(S,:) (the column Nystrom form, Section 1.2) and
    F(S,:) = chol(K(S,S)) for an arbitrary (not sampled) pivot order."""
    from oracle.pchol import pchol_given_pivots
    X = _pts(150, 3, 12)
    eps = 2.0
    K = kernel_dense(X, eps)
    S = np.random.Generator(np.random.PCG64(5)).permutation(150)[:30]
    rp = pchol_given_pivots(X, eps, S, blocks=[7, 1, 12, 10])
    F = rp["F"]
    KS = K[:, S]
    ny = KS @ np.linalg.solve(K[np.ix_(S, S)], KS.T)
    assert np.max(np.abs(F @ F.T - ny)) < 1e-10
    assert np.max(np.abs(F[S] - np.linalg.cholesky(K[np.ix_(S, S)]))) < 1e-12
    assert np.max(np.abs(rp["rho"] - np.maximum(np.diag(K - ny), 0))) < 1e-10


def test_replay_rejects_repeated_pivot():
    from oracle.pchol import pchol_given_pivots
    X = _pts(50, 3, 13)
    with pytest.raises(ValueError):
        pchol_given_pivots(X, 2.0, [3, 9, 3])
    with pytest.raises(ValueError):
        pchol_given_pivots(X, 2.0, [3, 9], blocks=[1])
