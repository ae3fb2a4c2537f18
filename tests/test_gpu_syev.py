"""GPU parity of the library's own top-k symmetric eigensolver (tridiagonal
reduction, bisection and inverse iteration, CholeskyQR2, ormtr), selected with
KEVD_SYEV=native, for the r x r EVD of Section 2 / Algorithm 1 (the default is
cuSOLVER's syevdx).

* Through the pipeline: eig_topk with the native solver against eig_topk with
  syevdx on the same d~, A, C, at the FP64 bars (eigenvalues 1e-10 relative,
  eigenvector clusters 1e-8).
* Against a construction: with F = I, d~ = 1 and A = I the route gives M = C and
  U = the eigenvectors of C, so C = Q diag(lambda) Q^T with chosen, partly
  repeated eigenvalues pins the values exactly and the cluster subspaces to Q.
"""
import os

import numpy as np
import pytest
import torch

from datagen import make_config
from oracle.pchol import arpc
from tests.helpers import compare_eigpairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kevd():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as m
    return m


def _eig(kevd, F, rk, dt, A, C, k, solver):
    old = os.environ.get("KEVD_SYEV")
    try:
        if solver == "native":
            os.environ["KEVD_SYEV"] = "native"
        else:
            os.environ.pop("KEVD_SYEV", None)
        ev, U, _ = kevd.eig_topk(F, rk, dt, A, C, k)
        return ev.cpu().numpy(), U.cpu().numpy().T
    finally:
        if old is None:
            os.environ.pop("KEVD_SYEV", None)
        else:
            os.environ["KEVD_SYEV"] = old


@pytest.mark.parametrize("N,r,b,k", [(3000, 64, 16, 8), (6000, 200, 50, 32), (5000, 333, 37, 96), (4000, 130, 65, 1)])
def test_native_matches_cusolver(kevd, N, r, b, k):
    X, eps, _ = make_config("ks200k", N=N)
    F = arpc(X, eps, r, b, 11)["F"]
    Fg = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    rk = F.shape[1]
    k = min(k, rk)
    dt, qt, A, C = kevd.bistoch_normalize(Fg, rk)
    ev_n, U_n = _eig(kevd, Fg, rk, dt, A, C, k, "native")
    ev_c, U_c = _eig(kevd, Fg, rk, dt, A, C, k, "cusolver")
    assert np.all(np.diff(ev_n) <= 0)
    erel, ang = compare_eigpairs(ev_c, U_c, ev_n, U_n)
    assert erel < 1e-10 and ang < 1e-8, (erel, ang)


def test_native_full_spectrum_norm_accuracy(kevd):
    """k = rank: the trailing eigenvalues of M fall to ~1e-10 of the leading one,
    where any backward-stable solver is accurate to ~eps |M| only; both solvers
    agree to 1e-13 |M| on every eigenvalue."""
    X, eps, _ = make_config("ks200k", N=5000)
    F = arpc(X, eps, 333, 37, 11)["F"]
    Fg = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    rk = F.shape[1]
    dt, qt, A, C = kevd.bistoch_normalize(Fg, rk)
    ev_n, _ = _eig(kevd, Fg, rk, dt, A, C, rk, "native")
    ev_c, _ = _eig(kevd, Fg, rk, dt, A, C, rk, "cusolver")
    assert np.max(np.abs(ev_n - ev_c)) < 1e-13 * np.max(np.abs(ev_c))


@pytest.mark.parametrize("solver", ["native", "cusolver"])
@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (40, 12), (300, 64), (700, 700)])
def test_constructed_spectrum(kevd, n, k, solver):
    rng = np.random.Generator(np.random.PCG64(n))
    # descending spectrum with exact repeats (a triple, pairs) over two decades
    base = np.sort(rng.uniform(1e-2, 1.0, n))[::-1].copy()
    if n >= 12:
        base[1:4] = base[1]          # triple
        base[5:7] = base[5]          # pair
        base[9:11] = base[9]         # pair
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    C = (Q * base) @ Q.T
    C = 0.5 * (C + C.T)
    I = torch.eye(n, dtype=torch.float64).cuda()
    dt = torch.ones(n, dtype=torch.float64).cuda()
    ev, U = _eig(kevd, I, n, dt, I.clone(), torch.from_numpy(np.ascontiguousarray(C.T)).cuda(), k, solver)
    lam = base[:k]
    assert np.max(np.abs(ev - lam) / lam) < 1e-10
    assert np.max(np.abs(U.T @ U - np.eye(k))) < 1e-12
    # cluster subspaces against the constructed eigenvectors
    _, ang = compare_eigpairs(lam, Q[:, :k], ev, U, lam_full=base)
    assert ang < 1e-8
    # residual of the eigen-equation
    assert np.max(np.abs(C @ U - U * ev)) < 1e-12 * max(1.0, base[0])
