"""GPU parity of bistoch_normalize and eig_topk (FP64) against the oracle's
Algorithm 1 (Householder QR route), and end to end against the dense P (-m gpu).

Tolerances (FP64 path): degree vectors and Gram matrices 1e-12 relative,
eigenvalues 1e-10 relative, eigenvector subspaces (clusters of eigenvalues with
relative gap < 1e-6 compared as subspaces) 1e-8 in the sine of the largest
principal angle.
"""
import numpy as np
import pytest
import torch

from datagen import make_config
from oracle.pchol import greedy_pchol, arpc
from oracle.alg1 import bistochastic_evd, degree_vectors
from oracle.kernel import kernel_dense
from oracle.dense import bistochastic_dense, top_eigh
from tests.helpers import compare_eigpairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kevd():
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as m
    return m


def _Fgpu(F):
    return torch.from_numpy(np.ascontiguousarray(F.T)).cuda()


def _check_normalize(kevd, F):
    rank = F.shape[1]
    dt, qt, A, C = kevd.bistoch_normalize(_Fgpu(F), rank)
    d0, q0 = degree_vectors(F)
    assert np.max(np.abs(dt.cpu().numpy() - d0) / np.abs(d0)) < 1e-12
    assert np.max(np.abs(qt.cpu().numpy() - q0) / np.abs(q0)) < 1e-12
    A0 = F.T @ (F / (d0 * d0)[:, None])
    C0 = F.T @ (F / q0[:, None])
    A = A.cpu().numpy()
    C = C.cpu().numpy()
    assert np.array_equal(A, A.T) and np.array_equal(C, C.T)
    assert np.max(np.abs(A - A0)) < 1e-12 * np.max(np.abs(A0))
    assert np.max(np.abs(C - C0)) < 1e-12 * np.max(np.abs(C0))
    return dt, qt


@pytest.mark.parametrize("case", ["ks2k_greedy", "arpc_ragged"])
def test_normalize_and_eig_match_alg1(kevd, case):
    if case == "ks2k_greedy":
        X, eps, _ = make_config("ks2k")
        F = greedy_pchol(X, eps, 128)[0]
        k = 32
    else:
        X, eps, _ = make_config("ks200k", N=3001)
        F = arpc(X, eps, 200, 40, 21)["F"]
        k = 40
    rank = F.shape[1]
    Fg = _Fgpu(F)
    dt, qt, A, C = kevd.bistoch_normalize(Fg, rank)
    _check_normalize(kevd, F)
    ev, U, kept = kevd.eig_topk(Fg, rank, dt, A, C, k)
    lam0, U0 = bistochastic_evd(F)
    ev = ev.cpu().numpy()
    U = U.cpu().numpy().T
    assert np.all(np.diff(ev) <= 0)
    erel, ang = compare_eigpairs(lam0[:k], U0[:, :k], ev, U, rel_gap=1e-6, lam_full=lam0)
    assert erel < 1e-10, erel
    assert ang < 1e-8, ang
    assert np.max(np.abs(U.T @ U - np.eye(k))) < 1e-10
    # sign convention: entry of largest magnitude is positive
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(k)] > 0)


def test_ks2k_end_to_end_vs_dense_P(kevd):
    """Config 1: greedy r=128 -> top-32 of P~, checked against the dense P."""
    X, eps, _ = make_config("ks2k")
    Xg = torch.from_numpy(X).cuda()
    out = kevd.rpchol_factor(Xg, eps, 128, mode="greedy")
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], out["rank"])
    ev, U, kept = kevd.eig_topk(out["F"], out["rank"], dt, A, C, 32)
    ev = ev.cpu().numpy()
    P, _, _ = bistochastic_dense(kernel_dense(X, eps))
    lamP, UP = top_eigh(P, 32)
    # approximation error of the method (not parity): the leading eigenvalues agree closely
    assert abs(ev[0] - 1.0) < 1e-8 and abs(lamP[0] - 1.0) < 1e-12
    assert np.max(np.abs(ev[:8] - lamP[:8])) < 1e-3
    # Theorem 4 holds for this factor
    from oracle.bounds import theorem4_bound
    F = out["F"].cpu().numpy().T
    a, b = theorem4_bound(kernel_dense(X, eps), F @ F.T)
    assert a <= b


def test_degree_not_positive(kevd):
    # rows 0 and 2 of F F^T sum to zero
    F = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]] + [[0.0, 1.0]] * 5)
    with pytest.raises(kevd.KevdError) as e:
        kevd.bistoch_normalize(_Fgpu(F), 2)
    assert e.value.status == 2


# FP64 Grams: with an even leading dimension (and F 16-byte aligned) the
# tensor-core kernel with exact digit-sliced products (gram_oz.cu) runs; an odd
# one, or KEVD_GRAM=fp64, the FP64-pipe kernel.  N = 3001 and 20,037 end in a
# partial 16-row quarter; rank 129 / 300 / 700 span several 128 x 64 tiles and
# leave ragged ones.
@pytest.mark.parametrize("N,rank,pad,gram", [(3001, 200, 1, None), (20000, 300, 0, None), (5000, 129, 3, None),
                                             (20037, 300, 1, None), (20000, 300, 0, "fp64"),
                                             (60000, 700, 0, None)])
def test_fp64_grams_tensor_core_and_fp64_pipe(kevd, monkeypatch, N, rank, pad, gram):
    """Both Gram matrices of an FP64 factor at the FP64 bar (1e-12 of the largest
    entry, exactly symmetric), and the one-Gram symmetric form."""
    if gram:
        monkeypatch.setenv("KEVD_GRAM", gram)
    X, eps, _ = make_config("ks200k" if rank < 500 else "vsa2m", N=N)
    F = arpc(X.astype(np.float64), eps, rank, 16 if rank < 500 else 100, 7)["F"]
    rk = F.shape[1]
    Fbuf = torch.full((rk, N + pad), float("nan"), dtype=torch.float64)
    Fbuf[:, :N] = torch.from_numpy(np.ascontiguousarray(F.T))
    Fg = Fbuf.cuda()[:, :N]
    dt, qt, A, C = kevd.bistoch_normalize(Fg, rk)
    d0, q0 = degree_vectors(F)
    A0 = F.T @ (F / (d0 * d0)[:, None])
    C0 = F.T @ (F / q0[:, None])
    A = A.cpu().numpy()
    C = C.cpu().numpy()
    assert np.array_equal(A, A.T) and np.array_equal(C, C.T)
    assert np.max(np.abs(A - A0)) < 1e-12 * np.max(np.abs(A0))
    assert np.max(np.abs(C - C0)) < 1e-12 * np.max(np.abs(C0))
    for G, G0 in ((A, A0), (C, C0)):
        assert abs(np.mean((np.diag(G) - np.diag(G0)) / np.diag(G0))) < 1e-13
    ds, As = kevd.symmetric_normalize(Fg, rk)
    As0 = F.T @ (F / d0[:, None])
    As = As.cpu().numpy()
    assert np.array_equal(As, As.T)
    assert np.max(np.abs(As - As0)) < 1e-12 * np.max(np.abs(As0))
