"""Planted mistakes in the oracle (on the CPU) must trip its pins.

Each case copies one oracle module, applies a plausible one-token mistake (a
dropped term, a wrong sign, a transposed operand, a wrong index rule), and
checks that the corresponding pin fails on the mutant while passing on the
original.
"""
import inspect
import types

import numpy as np
import pytest

import oracle.alg1
import oracle.pchol
from oracle.kernel import kernel_dense
from oracle.dense import lowrank_bistochastic_dense, top_eigh


def _mutant(mod, old, new):
    src = inspect.getsource(mod)
    assert old in src, old
    m = types.ModuleType(mod.__name__ + "_mutant")
    m.__package__ = "oracle"
    exec(compile(src.replace(old, new), m.__name__, "exec"), m.__dict__)
    return m


def _pts(n, d, seed=0):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, d))


def _alg1_pin(mod):
    X = _pts(120, 3, 1)
    F = oracle.pchol.greedy_pchol(X, 4.0, 20)[0]
    lam, U = mod.bistochastic_evd(F, k=8)
    Pt, _, _ = lowrank_bistochastic_dense(F)
    lam_d, _ = top_eigh(Pt, 8)
    return np.max(np.abs(lam - lam_d)) < 1e-10 and np.max(np.abs(Pt @ U - U * lam)) < 1e-10


ALG1_MUTANTS = [
    ("F / q[:, None]", "F * q[:, None]"),                 # wrong inner weight
    ("R1 @ C @ R1.T", "R1.T @ C @ R1"),                   # transposed operand
    ("F / d[:, None], mode", "F / np.sqrt(d)[:, None], mode"),  # wrong outer scaling
    ("F.T @ (1.0 / d)", "F.T @ d"),                       # dropped inverse
]


@pytest.mark.parametrize("old,new", ALG1_MUTANTS)
def test_alg1_mutants_fail_pins(old, new):
    assert _alg1_pin(oracle.alg1)
    assert not _alg1_pin(_mutant(oracle.alg1, old, new))


def _pchol_pin(mod):
    X = _pts(200, 3, 2)
    eps = 3.0
    K = kernel_dense(X, eps)
    ok = True
    # greedy against dense Schur complement brute force
    F, S, rho, _ = mod.greedy_pchol(X, eps, 25)
    E = K.copy()
    piv = []
    for _ in range(25):
        s = int(np.argmax(np.diag(E)))
        piv.append(s)
        E = E - np.outer(E[:, s], E[s, :]) / E[s, s]
    ok &= S.tolist() == piv
    # ARPC: residual diagonal, PSD order and Nystrom identity
    out = mod.arpc(X, eps, 48, 12, seed=4)
    F, S, rho = out["F"], out["pivots"], out["rho"]
    R = K - F @ F.T
    ok &= np.max(np.abs(rho - np.maximum(np.diag(R), 0))) < 1e-10
    ok &= np.linalg.eigvalsh(R).min() > -1e-10
    Kn = K[:, S] @ np.linalg.pinv(K[np.ix_(S, S)], rcond=1e-13) @ K[S, :]
    ok &= np.max(np.abs(Kn - F @ F.T)) < 1e-8
    # sampling law
    rho = np.array([1.0, 3.0, 0.5, 0.0, 2.5, 1.0])
    u = np.linspace(0, 1, 4001)[:-1] + 1 / 8000
    j, _ = mod.inverse_cdf(rho, u)
    ok &= np.allclose(np.bincount(j, minlength=6) / 4000, rho / rho.sum(), atol=1e-3)
    # exact CDF edges: u * sum = cumsum_j must pick the next index with rho > 0
    c = np.cumsum(rho)
    j, _ = mod.inverse_cdf(rho, c[:-1] / c[-1])
    ok &= j.tolist() == [1, 2, 4, 4, 5]
    # reject law: H = [[1, .6], [.6, 1]], second accepted with probability 0.64
    H = np.array([[1.0, 0.6], [0.6, 1.0]])
    acc = sum(1 in mod.reject(H, np.array([0.1, z]))[0].tolist() for z in np.linspace(0, 1, 1001)[:-1])
    ok &= abs(acc / 1000 - 0.64) < 2e-3
    return bool(ok)


PCHOL_MUTANTS = [
    ("rho - np.sum(G * G, axis=1)", "rho + np.sum(G * G, axis=1)"),        # wrong sign
    ("solve_triangular(L, R.T, lower=True).T", "solve_triangular(L.T, R.T, lower=False).T"),
    ("z[i] * rho0[i] < H[i, i]", "z[i] * H[i, i] < rho0[i]"),              # swapped reject test
    ('side="right"', 'side="left"'),                                        # CDF edge rule
    ("- F[:, :k] @ F[acc, :k].T", "- F[:, :k] @ F[acc, :k].T * 0"),         # dropped overlap term
    ("H[i + 1:, i + 1:] -= np.outer", "H[i + 1:, i + 1:] += np.outer"),    # Schur sign
    ("s = int(np.argmax(rho))", "s = int(np.argmax(rho[::-1]))"),          # wrong index
]


@pytest.mark.parametrize("old,new", PCHOL_MUTANTS)
def test_pchol_mutants_fail_pins(old, new):
    assert _pchol_pin(oracle.pchol)
    try:
        ok = _pchol_pin(_mutant(oracle.pchol, old, new))
    except (np.linalg.LinAlgError, ValueError, IndexError, FloatingPointError):
        ok = False
    assert not ok


def _lowmem_pin(mod):
    """The low-memory oracle against the pinned ARPC and Algorithm 1 oracles and the dense K."""
    X = _pts(300, 3, 5)
    eps = 3.0
    ref = oracle.pchol.arpc(X, eps, 60, 12, seed=9)
    low = mod.arpc_lowmem(X, eps, 60, 12, seed=9, panel=70)
    S, W = low["pivots"], low["W"]
    ok = S.tolist() == ref["pivots"].tolist()
    ok &= np.max(np.abs(low["rho"] - ref["rho"])) < 1e-10
    K = kernel_dense(X, eps)
    if len(S) == len(ref["pivots"]):
        ok &= np.max(np.abs(W @ W.T - K[np.ix_(S, S)])) < 1e-10
        F = mod.lowmem_rows(X, eps, S, W, np.arange(300))
        ok &= np.max(np.abs(F - ref["F"])) < 1e-8
    F = ref["F"]
    d0, q0 = oracle.alg1.degree_vectors(F)
    dt, qt, A, C = mod.normalize_lowmem(X, eps, ref["pivots"], F[ref["pivots"]], panel=70)
    ok &= np.max(np.abs(dt - d0) / d0) < 1e-10 and np.max(np.abs(qt - q0) / q0) < 1e-10
    ok &= np.max(np.abs(A - F.T @ (F / (d0 ** 2)[:, None]))) < 1e-10 * np.max(np.abs(A))
    lam0, U0 = oracle.alg1.bistochastic_evd(F, k=6)
    lam, U = mod.evd_lowmem(X, eps, ref["pivots"], F[ref["pivots"]], 6, panel=70)
    ok &= np.max(np.abs(lam - lam0) / np.abs(lam0)) < 1e-10
    ok &= np.max(np.abs(np.abs(np.sum(U * U0, axis=0)) - 1.0)) < 1e-8
    return bool(ok)


LOWMEM_MUTANTS = [
    ("return solve_triangular(W, Kc.T, lower=True).T", "return solve_triangular(W.T, Kc.T, lower=False).T"),
    ("R = R - kernel_block(X[i0:i1], X[S], eps) @ Z", "R = R + kernel_block(X[i0:i1], X[S], eps) @ Z"),
    ("Z = solve_triangular(W.T, solve_triangular(", "Z = (lambda A, B, lower: B)(W.T, solve_triangular("),  # dropped W^-T
    ("Wn[k:, :k] = Fp[T]", "Wn[k:, :k] = Fp[: len(T)]"),                     # wrong rows of F(S',:)
    ("qt[i0:i1] = Fp @ t", "qt[i0:i1] = Fp @ s"),                            # wrong vector
    ("(dt[i0:i1] ** 2)[:, None]", "dt[i0:i1][:, None]"),                     # dropped square
    ("Y = solve_triangular(R, V, lower=False)", "Y = V"),                    # dropped R^-1
]


@pytest.mark.parametrize("old,new", LOWMEM_MUTANTS)
def test_lowmem_mutants_fail_pins(old, new):
    import oracle.lowmem
    assert _lowmem_pin(oracle.lowmem)
    try:
        ok = _lowmem_pin(_mutant(oracle.lowmem, old, new))
    except (np.linalg.LinAlgError, ValueError, IndexError, FloatingPointError):
        ok = False
    assert not ok


import oracle.bounds


def _bounds_pin(mod):
    """The hand-derived two-point Nystrom case of tests/test_oracle_bounds.py."""
    from tests.test_oracle_bounds import K as K2, KT as KT2
    ok = abs(mod.theorem2_bound(K2, KT2)[1] - 56.7029003976) < 1e-8
    ok &= abs(mod.theorem4_bound(K2, KT2)[1] - 624.0213249359) < 1e-7
    ok &= abs(mod.lemma_qbound(K2, KT2)[1] - 15.0 * np.sqrt(2.0)) < 1e-12
    ok &= abs(mod.lemma_dbound(K2, KT2)[1] - np.sqrt(2.0) * 15.0 / 16.0) < 1e-12
    return bool(ok)


BOUNDS_MUTANTS = [
    ("br = (1 / (np.sqrt(qmin) * dmin) + np.sqrt(N) * trK", "br = (1 / (np.sqrt(qmin) * dmin) + trK"),  # dropped sqrt(N)
    ("br = (1 / (np.sqrt(qmin) * dmin)", "br = (1 / (np.sqrt(qmin) * dd)"),     # delta_d for d_min
    ("pref * br * tr", "pref ** 2 * br * tr"),                                 # (1 + |G~|) squared
    ("(1 + normK / dd))", "(1 + normK / dmin))"),                             # d_min for delta_d
    ("np.sqrt(N) / delta_d * (1 + normK", "N / delta_d * (1 + normK"),        # N for sqrt(N)
    ("delta_d = min(d.min(), dt.min())", "delta_d = d.min()"),                # d_min for delta_d
    ("b = (1 / dmin + np.sqrt(N) / delta ** 2", "b = (1 / delta + np.sqrt(N) / delta ** 2"),  # delta for d_min
    ("N / (4 * delta ** 3)", "N / (4 * delta ** 2)"),                          # wrong power
    ("np.sqrt(N) * tr, np.sum", "N * tr, np.sum"),                             # Lemma dbound: N for sqrt(N)
]


@pytest.mark.parametrize("old,new", BOUNDS_MUTANTS)
def test_bounds_mutants_fail_pins(old, new):
    assert _bounds_pin(oracle.bounds)
    assert not _bounds_pin(_mutant(oracle.bounds, old, new))


def _replay_pin(mod):
    from tests.test_oracle_pchol import test_replay_is_nystrom_and_cholesky_of_pivot_block as pin
    saved = oracle.pchol.pchol_given_pivots
    oracle.pchol.pchol_given_pivots = mod.pchol_given_pivots
    try:
        pin()
        return True
    except (AssertionError, ValueError):     # a failed pin, or H no longer positive definite
        return False
    finally:
        oracle.pchol.pchol_given_pivots = saved


REPLAY_MUTANTS = [
    ("H = kernel_block(X[T], X[T], eps) - F[T, :k] @ F[T, :k].T", "H = kernel_block(X[T], X[T], eps)"),  # dropped Schur
    ("R = kernel_columns(X, T, eps) - F[:, :k] @ F[T, :k].T", "R = kernel_columns(X, T, eps) + F[:, :k] @ F[T, :k].T"),
    ("G = solve_triangular(L, R.T, lower=True).T          # R L^-T\n        F[:, k:k + m] = G\n        rho",
     "G = solve_triangular(L.T, R.T, lower=False).T\n        F[:, k:k + m] = G\n        rho"),            # L^-1 for L^-T
]


@pytest.mark.parametrize("old,new", REPLAY_MUTANTS)
def test_replay_mutants_fail_pins(old, new):
    assert _replay_pin(oracle.pchol)
    assert not _replay_pin(_mutant(oracle.pchol, old, new))
