"""Pivoted partial Cholesky of an implicit kernel matrix (Section 1.2, Appendix A).

* greedy_pchol -- pivot s = argmax of the residual diagonal rho (the
  deterministic extreme of RPC described in Appendix A), one pivot per step.
* arpc         -- Algorithm 2 (accelerated randomly pivoted Cholesky) with the
  accept/reject check of Algorithm 3.
The residual diagonal rho = diag(K - F F^T) starts at diag(K) (= 1 for the
Gaussian kernel), loses rownorms(G)^2 after each block and is clamped at 0.

Readings where the paper is silent or garbled:
* Algorithm 2's sampling line names the law d/sum(d); the text of Appendix A
  defines it as rho/sum(rho), used here, with zero-based proposal indices.
* Proposals are the inverse CDF of rho: the smallest j with cumsum(rho)_j >
  u * sum(rho), u from Philox stream 0; draw order is the reject order.
* Algorithm 3 accepts proposal i iff z * rho0(i) < H(i,i) with rho0 = diag(H)
  taken before the loop, z from Philox stream 1; a proposal whose current
  H(i,i) is not positive is rejected (guards rounding; duplicates of an
  accepted pivot have H(i,i)=0 in exact arithmetic).
* t = r/b rounds (F has at most r columns).  until_rank=True keeps drawing
  rounds, truncating the last one, until exactly r pivots are accepted.
* If sum(rho) reaches 0 the remaining rounds are skipped.
* Greedy: ties go to the lowest index; H = K(s,s) - |F(s,:)|^2 is recomputed
  from F (Algorithm 2 with b=1 and no rejection); stop when H <= 0.
"""
import numpy as np
from scipy.linalg import solve_triangular

from .kernel import kernel_columns, kernel_block
from .philox import uniforms, STREAM_PROPOSE, STREAM_REJECT


def inverse_cdf(rho, u):
    """Indices j = min{j : cumsum(rho)_j > u * sum(rho)} and their relative margins.

    The margin of a draw is the distance of u*sum(rho) to the nearer edge of the
    chosen CDF interval, divided by sum(rho): draws with a tiny margin may pick a
    neighbouring index under another summation order.
    """
    c = np.cumsum(rho)
    total = c[-1]
    t = np.asarray(u) * total
    j = np.searchsorted(c, t, side="right")
    last = int(np.flatnonzero(rho > 0)[-1])
    j = np.minimum(j, last)
    lo = np.where(j > 0, c[np.maximum(j - 1, 0)], 0.0)
    margin = np.minimum(c[j] - t, t - lo) / total
    return j.astype(np.int64), margin


def reject(H, z):
    """Algorithm 3: accepted positions T (into the proposal list) and L = chol(H(T,T))."""
    H = np.array(H, dtype=np.float64, copy=True)
    b = H.shape[0]
    L = np.zeros((b, b))
    T = []
    rho0 = np.diag(H).copy()
    margins = np.empty(b)
    for i in range(b):
        margins[i] = H[i, i] - z[i] * rho0[i]
        if H[i, i] > 0 and z[i] * rho0[i] < H[i, i]:
            T.append(i)
            L[i:, i] = H[i:, i] / np.sqrt(H[i, i])
            H[i + 1:, i + 1:] -= np.outer(L[i + 1:, i], L[i + 1:, i])
    T = np.array(T, dtype=np.int64)
    return T, L[np.ix_(T, T)], margins


def greedy_pchol(X, eps, r):
    """Greedy pivoted partial Cholesky to rank <= r.

    Returns (F N x rank, pivots, rho, rho_history) where rho_history[i] is
    sum(rho) after i pivots.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    F = np.zeros((N, r))
    rho = np.ones(N)               # diag K = k(x, x) = 1
    piv = []
    hist = [rho.sum()]
    for i in range(r):
        s = int(np.argmax(rho))    # first maximum = lowest index on ties
        if rho[s] <= 0:
            break
        col = kernel_columns(X, [s], eps)[:, 0]
        H = col[s] - F[s, :i] @ F[s, :i]
        if H <= 0:
            break
        g = (col - F[:, :i] @ F[s, :i]) / np.sqrt(H)
        F[:, i] = g
        piv.append(s)
        rho = np.maximum(rho - g * g, 0.0)
        hist.append(rho.sum())
    k = len(piv)
    return F[:, :k], np.array(piv, dtype=np.int64), rho, np.array(hist)


def arpc(X, eps, r, b, seed, until_rank=False, max_rounds=None):
    """Algorithm 2 (ARPC).  Returns a dict with F (N x rank), pivots, rho and a per-round log.

    The log holds, for round i: proposals, their inverse-CDF margins, the
    accepted positions, the reject margins and sum(rho) before the round.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    F = np.zeros((N, r))
    rho = np.ones(N)
    piv = []
    k = 0
    t = r // b
    if max_rounds is None:
        max_rounds = t if not until_rank else 8 * t + 64
    log = []
    rnd = 0
    while rnd < max_rounds and k < r:
        if not until_rank and rnd >= t:
            break
        total = rho.sum()
        if not total > 0:
            break
        u = uniforms(seed, STREAM_PROPOSE, rnd, b)
        prop, pmargin = inverse_cdf(rho, u)
        H = kernel_block(X[prop], X[prop], eps) - F[prop, :k] @ F[prop, :k].T
        z = uniforms(seed, STREAM_REJECT, rnd, b)
        T, L, rmargin = reject(H, z)
        if k + len(T) > r:                     # until_rank: truncate the last round
            T = T[: r - k]
            L = L[: len(T), : len(T)]
        m = len(T)
        log.append(dict(proposals=prop, prop_margin=pmargin, accepted=T,
                        reject_margin=rmargin, sum_rho=total))
        if m:
            acc = prop[T]
            R = kernel_columns(X, acc, eps) - F[:, :k] @ F[acc, :k].T
            G = solve_triangular(L, R.T, lower=True).T          # R L^-T
            F[:, k:k + m] = G
            k += m
            piv.extend(acc.tolist())
            rho = np.maximum(rho - np.sum(G * G, axis=1), 0.0)
        rnd += 1
    return dict(F=F[:, :k], pivots=np.array(piv, dtype=np.int64), rho=rho, rounds=rnd, log=log)


def pchol_given_pivots(X, eps, S, blocks=None):
    """Partial Cholesky factor for a given accepted pivot sequence (replay).

    Runs Algorithm 2's column update in FP64 with the pivots fixed instead of
    drawn: for each block T of consecutive pivots (``blocks`` = block lengths,
    default one pivot per block), H = K(T,T) - F(T,:) F(T,:)^T, L = chol(H)
    (Algorithm 3 with every proposal accepted), G = (K(:,T) - F F(T,:)^T) L^-T,
    F gains the columns G and rho loses rownorms(G)^2 (clamped at 0).  Column j
    of F depends only on S[0..j], so the block grouping changes rounding only.
    Used to score a factor whose pivots came from another arithmetic (the
    precision form) against the FP64 factor of the same pivots.

    Returns dict(F N x len(S), rho).  Raises ValueError if some H is not
    positive definite (a pivot repeated, or numerically dependent).
    """
    X = np.asarray(X, dtype=np.float64)
    S = np.asarray(S, dtype=np.int64)
    N, r = X.shape[0], len(S)
    if blocks is None:
        blocks = [1] * r
    if sum(blocks) != r:
        raise ValueError("block lengths do not add up to the number of pivots")
    F = np.zeros((N, r))
    rho = np.ones(N)
    k = 0
    for m in blocks:
        T = S[k:k + m]
        H = kernel_block(X[T], X[T], eps) - F[T, :k] @ F[T, :k].T
        try:
            L = np.linalg.cholesky(H)
        except np.linalg.LinAlgError as e:
            raise ValueError("H of pivots %s is not positive definite" % T.tolist()) from e
        R = kernel_columns(X, T, eps) - F[:, :k] @ F[T, :k].T
        G = solve_triangular(L, R.T, lower=True).T          # R L^-T
        F[:, k:k + m] = G
        rho = np.maximum(rho - np.sum(G * G, axis=1), 0.0)
        k += m
    return dict(F=F, rho=rho)
