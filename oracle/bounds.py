"""Error bounds of Section 3 and Appendix B, evaluated densely (tiny N).

Used by the tests to pin the oracle: every quantity below is a dense
definition from the paper's statements.
"""
import numpy as np


def trace_norm(M):
    """Trace (nuclear) norm of a symmetric matrix: sum of |eigenvalues|."""
    return float(np.sum(np.abs(np.linalg.eigvalsh(M))))


def lemma_dbound(K, Kt):
    """Lemma dbound: (max|d-d~|, sqrt(N) tr(K-K~), sum (d-d~)^2, N tr(K-K~)^2)."""
    N = K.shape[0]
    d = K.sum(1)
    dt = Kt.sum(1)
    tr = np.trace(K - Kt)
    return np.max(np.abs(d - dt)), np.sqrt(N) * tr, np.sum((d - dt) ** 2), N * tr ** 2


def lemma_qbound(K, Kt):
    """Lemma qbound: (max|q-q~|, sqrt(N)/delta_d (1 + |K|/delta_d) tr(K-K~))."""
    N = K.shape[0]
    d = K.sum(1)
    dt = Kt.sum(1)
    q = K @ (1 / d)
    qt = Kt @ (1 / dt)
    delta_d = min(d.min(), dt.min())
    normK = np.linalg.norm(K, 2)
    tr = np.trace(K - Kt)
    return np.max(np.abs(q - qt)), np.sqrt(N) / delta_d * (1 + normK / delta_d) * tr


def theorem4_bound(K, Kt):
    """Theorem 4: (|P - P~|_*, bound).  G~ = Q~^-1/2 K~ D~^-1 (Eq. (gram))."""
    N = K.shape[0]
    one = np.ones(N)
    d = K @ one
    q = K @ (1 / d)
    dt = Kt @ one
    qt = Kt @ (1 / dt)
    P = (K / d[:, None]) @ (K / (q[:, None] * d[None, :]))
    Pt = (Kt / dt[:, None]) @ (Kt / (qt[:, None] * dt[None, :]))
    Gt = (Kt / np.sqrt(qt)[:, None]) / dt[None, :]
    dmin, qmin = d.min(), q.min()
    dd = min(dmin, dt.min())
    dq = min(qmin, qt.min())
    trK = np.trace(K)
    normK = np.linalg.norm(K, 2)
    tr = np.trace(K - Kt)
    pref = 1 + np.linalg.norm(Gt, 2)
    br = (1 / (np.sqrt(qmin) * dmin) + np.sqrt(N) * trK / (np.sqrt(dq) * dd ** 2)
          + np.sqrt(N) * trK / (2 * dq ** 1.5 * dd ** 2) * (1 + normK / dd))
    return trace_norm(P - Pt), pref * br * tr


def theorem2_bound(K, Kt):
    """Theorem 2 (symmetric normalisation): (|L - L~|_*, bound)."""
    N = K.shape[0]
    d = K.sum(1)
    dt = Kt.sum(1)
    L = K / np.sqrt(np.outer(d, d))
    Lt = Kt / np.sqrt(np.outer(dt, dt))
    dmin = d.min()
    delta = min(dmin, dt.min())
    trK = np.trace(K)
    tr = np.trace(K - Kt)
    b = (1 / dmin + np.sqrt(N) / delta ** 2 * trK + N / (4 * delta ** 3) * trK * tr) * tr
    return trace_norm(L - Lt), b


def theorem1_rank(r_prime, eps_rel, eta):
    """Smallest r allowed by Theorem 1: r >= r'/eps + r' log(1/(eps eta))."""
    return r_prime / eps_rel + r_prime * np.log(1 / (eps_rel * eta))


def best_rank_error(K, r_prime):
    """tr(K - [K]_r') = sum of the trailing N - r' eigenvalues of K."""
    lam = np.sort(np.linalg.eigvalsh(K))[::-1]
    return float(np.sum(lam[r_prime:]))
