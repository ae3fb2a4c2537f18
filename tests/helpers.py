"""Comparison helpers shared by the parity tests (test infrastructure)."""
import numpy as np


def max_angle(U, V):
    """sin of the largest principal angle between the column spaces of U and V."""
    Qu, _ = np.linalg.qr(np.asarray(U, dtype=np.float64))
    Qv, _ = np.linalg.qr(np.asarray(V, dtype=np.float64))
    return float(np.linalg.norm(Qv - Qu @ (Qu.T @ Qv), 2))


def clusters(lam, rel_gap):
    """Groups of consecutive (descending) eigenvalues whose relative gap is < rel_gap."""
    groups = [[0]]
    for i in range(1, len(lam)):
        gap = abs(lam[i - 1] - lam[i]) / max(abs(lam[i - 1]), 1e-300)
        if gap < rel_gap:
            groups[-1].append(i)
        else:
            groups.append([i])
    return groups


def compare_eigpairs(lam_ref, U_ref, lam, U, rel_gap=1e-6, lam_full=None):
    """(max relative eigenvalue error, max cluster subspace angle).

    Clusters are formed on the reference eigenvalues; a cluster touching the
    last index is skipped when the next reference eigenvalue (lam_full) would
    belong to it (the k cut splits it).
    """
    lam_ref = np.asarray(lam_ref)
    lam = np.asarray(lam)
    erel = float(np.max(np.abs(lam - lam_ref) / np.abs(lam_ref)))
    worst = 0.0
    k = len(lam_ref)
    for g in clusters(lam_ref, rel_gap):
        if g[-1] == k - 1 and lam_full is not None and len(lam_full) > k:
            nxt = lam_full[k]
            if abs(lam_ref[-1] - nxt) / abs(lam_ref[-1]) < rel_gap:
                continue
        worst = max(worst, max_angle(U_ref[:, g], U[:, g]))
    return erel, worst


def first_divergence(a, b):
    a, b = list(a), list(b)
    for i, (x, y) in enumerate(zip(a, b)):
        if x != y:
            return i
    return None if len(a) == len(b) else min(len(a), len(b))
