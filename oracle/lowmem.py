"""Low-memory ARPC and the bistochastic EVD from its factor (test infrastructure).

Appendix A (its closing paragraph) and the Remark of Section 4.2 note that ARPC
can keep only an r x r factor of F and recompute the other entries when they
are needed, which removes the N x r factor from memory.  This module is that variant, written from the
mathematics of the paper, for checking a device implementation against.

Representation: the accepted pivots S (acceptance order) and W = F(S,:), the
k x k block of the factor at the pivot rows, lower triangular.  Because
F F^T = K(:,S) K(S,S)^-1 K(S,:) (the Nystrom form of Section 1.2) and
W W^T = K(S,S), every row of F is F(i,:) = K(i,S) W^-T: one kernel row and a
triangular solve.  Whole passes over F become passes over K(:,S), computed
from X in row panels of `panel` rows, so no array with N x r entries exists.

* arpc_lowmem      -- Algorithm 2 with Algorithm 3, F replaced by (S, W).
* lowmem_rows      -- F(rows,:) from (S, W).
* normalize_lowmem -- d~, q~ and the Grams A = F^T D~^-2 F, C = F^T Q~^-1 F
                      (Algorithm 1's degree vectors and the B C B^T form of
                      Section 2) in three passes, F rebuilt in each.
* evd_lowmem       -- top-k eigenpairs of P~ from A and C (Cholesky of A,
                      EVD of R C R^T) and the lift U = D~^-1 F Y.
The device code may form the vectors K(:,S) (W^-T v) directly; the oracle
always rebuilds F, the plain definition.
"""
import numpy as np
from scipy.linalg import solve_triangular, cholesky, eigh

from .kernel import kernel_block
from .philox import uniforms, STREAM_PROPOSE, STREAM_REJECT
from .pchol import inverse_cdf, reject
from .alg1 import NotPositive


def _panels(N, panel):
    for i0 in range(0, N, panel):
        yield i0, min(N, i0 + panel)


def lowmem_rows(X, eps, S, W, rows):
    """F(rows, :) = K(rows, S) W^-T."""
    X = np.asarray(X, dtype=np.float64)
    S = np.asarray(S, dtype=np.int64)
    if len(S) == 0:
        return np.zeros((len(rows), 0))
    Kc = kernel_block(X[rows], X[S], eps)
    return solve_triangular(W, Kc.T, lower=True).T


def arpc_lowmem(X, eps, r, b, seed, until_rank=False, max_rounds=None, panel=4096):
    """Algorithm 2 (ARPC) keeping only the pivots S and W = F(S,:).

    Each round: proposals from rho; F(S',:) = K(S',S) W^-T for the proposals;
    H = K(S',S') - F(S',:) F(S',:)^T; Algorithm 3 gives the accepted T and
    L = chol(H(T,T)); for every row, in panels,
    G = (K(:,T) - K(:,S) Z) L^-T with Z = W^-T W^-1 K(S,T) (that is, F F(T,:)^T),
    rho -= rownorms(G)^2 and clamp; then W grows by [F(T,:), L].
    Returns pivots, W, rho, rounds and the same per-round log as arpc.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    rho = np.ones(N)
    S = np.zeros(0, dtype=np.int64)
    W = np.zeros((0, 0))
    t = r // b
    if max_rounds is None:
        max_rounds = t if not until_rank else 8 * t + 64
    log = []
    rnd = 0
    while rnd < max_rounds and len(S) < r:
        k = len(S)
        if not until_rank and rnd >= t:
            break
        total = rho.sum()
        if not total > 0:
            break
        u = uniforms(seed, STREAM_PROPOSE, rnd, b)
        prop, pmargin = inverse_cdf(rho, u)
        Fp = lowmem_rows(X, eps, S, W, prop)                              # b x k
        H = kernel_block(X[prop], X[prop], eps) - Fp @ Fp.T
        z = uniforms(seed, STREAM_REJECT, rnd, b)
        T, L, rmargin = reject(H, z)
        if k + len(T) > r:                                                # until_rank: truncate the last round
            T = T[: r - k]
            L = L[: len(T), : len(T)]
        m = len(T)
        log.append(dict(proposals=prop, prop_margin=pmargin, accepted=T, reject_margin=rmargin, sum_rho=total))
        if m:
            acc = prop[T]
            if k:
                Z = solve_triangular(W.T, solve_triangular(W, kernel_block(X[S], X[acc], eps), lower=True),
                                     lower=False)                         # k x m: W^-T W^-1 K(S, T)
            for i0, i1 in _panels(N, panel):
                R = kernel_block(X[i0:i1], X[acc], eps)
                if k:
                    R = R - kernel_block(X[i0:i1], X[S], eps) @ Z
                G = solve_triangular(L, R.T, lower=True).T                # R L^-T
                rho[i0:i1] = np.maximum(rho[i0:i1] - np.sum(G * G, axis=1), 0.0)
            Wn = np.zeros((k + m, k + m))
            Wn[:k, :k] = W
            Wn[k:, :k] = Fp[T]
            Wn[k:, k:] = L
            W = Wn
            S = np.concatenate([S, acc])
        rnd += 1
    return dict(pivots=S, W=W, rho=rho, rounds=rnd, log=log)


def normalize_lowmem(X, eps, S, W, panel=4096):
    """(d~, q~, A, C) of Algorithm 1 / Section 2 with F rebuilt panel by panel.

    Three passes over the rows, each rebuilding F(rows,:) = K(rows,S) W^-T:
    pass 1 s = F^T 1; pass 2 d~ = F s and t = F^T d~^-1; pass 3 q~ = F t,
    A = F^T D~^-2 F and C = F^T Q~^-1 F (B = D~^-1 F, Section 2.2).  Raises
    NotPositive as Algorithm 1's asserts do.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    k = len(S)
    s = np.zeros(k)
    for i0, i1 in _panels(N, panel):
        s += lowmem_rows(X, eps, S, W, np.arange(i0, i1)).sum(axis=0)
    dt = np.empty(N)
    t = np.zeros(k)
    for i0, i1 in _panels(N, panel):
        Fp = lowmem_rows(X, eps, S, W, np.arange(i0, i1))
        dt[i0:i1] = Fp @ s
        if not np.all(dt[i0:i1] > 0):
            raise NotPositive("diag(D~) not positive")
        t += Fp.T @ (1.0 / dt[i0:i1])
    qt = np.empty(N)
    A = np.zeros((k, k))
    C = np.zeros((k, k))
    for i0, i1 in _panels(N, panel):
        Fp = lowmem_rows(X, eps, S, W, np.arange(i0, i1))
        qt[i0:i1] = Fp @ t
        if not np.all(qt[i0:i1] > 0):
            raise NotPositive("diag(Q~) not positive")
        A += Fp.T @ (Fp / (dt[i0:i1] ** 2)[:, None])
        C += Fp.T @ (Fp / qt[i0:i1][:, None])
    return dt, qt, A, C


def evd_lowmem(X, eps, S, W, k, panel=4096):
    """Top-k eigenpairs of P~ = B C B^T (B = D~^-1 F) with F rebuilt panel by
    panel: A = R^T R, M = R C R^T = V Lambda V^T, U = B R^-1 V (rows of U from
    the rows of F).  Eigenvalues descending; U is N x k."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    dt, qt, A, C = normalize_lowmem(X, eps, S, W, panel)
    R = cholesky(A, lower=False)
    M = R @ C @ R.T
    lam, V = eigh(0.5 * (M + M.T))
    order = np.argsort(lam)[::-1][:k]
    lam, V = lam[order], V[:, order]
    Y = solve_triangular(R, V, lower=False)                    # R^-1 V
    U = np.empty((N, k))
    for i0, i1 in _panels(N, panel):
        U[i0:i1] = (lowmem_rows(X, eps, S, W, np.arange(i0, i1)) @ Y) / dt[i0:i1, None]
    return lam, U
