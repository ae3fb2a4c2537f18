"""GPU parity of the symmetric normalisation (Section 2.1) and of the optional
constant-eigenvector fix of Algorithm 1, against the oracle (-m gpu)."""
import numpy as np
import pytest
import torch

from datagen import make_config
from oracle.pchol import arpc, greedy_pchol
from oracle.alg1 import symmetric_evd, constant_eigvec_fix
from tests.helpers import compare_eigpairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kevd():
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as m
    return m


@pytest.mark.parametrize("case", ["greedy", "arpc"])
def test_symmetric_fp64_matches_oracle(kevd, case):
    if case == "greedy":
        X, eps, _ = make_config("ks2k")
        F = greedy_pchol(X, eps, 128)[0]
        k = 32
    else:
        X, eps, _ = make_config("ks200k", N=4001)
        F = arpc(X, eps, 192, 32, 4)["F"]
        k = 24
    rank = F.shape[1]
    Fg = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    dt, As = kevd.symmetric_normalize(Fg, rank)
    d0 = F @ (F.T @ np.ones(F.shape[0]))
    assert np.max(np.abs(dt.cpu().numpy() - d0) / d0) < 1e-12
    A0 = F.T @ (F / d0[:, None])
    As = As.cpu().numpy()
    assert np.array_equal(As, As.T) and np.max(np.abs(As - A0)) < 1e-12 * np.max(np.abs(A0))
    ev, U = kevd.symmetric_eig_topk(Fg, rank, dt, torch.from_numpy(As).cuda(), k)
    lam0, U0 = symmetric_evd(F)
    erel, ang = compare_eigpairs(lam0[:k], U0[:, :k], ev.cpu().numpy(), U.cpu().numpy().T, rel_gap=1e-6,
                                 lam_full=lam0)
    assert erel < 1e-10 and ang < 1e-8, (erel, ang)
    assert abs(ev[0].item() - 1.0) < 1e-10        # L~ has eigenvalue 1 (eigenvector D~^1/2 1)


def test_symmetric_fp32_eigenvalues(kevd):
    X, eps, _ = make_config("ks200k", N=6000)
    F = arpc(X, eps, 256, 64, 8)["F"]
    F32 = np.ascontiguousarray(F.T, dtype=np.float32)
    rank = F.shape[1]
    Fg = torch.from_numpy(F32).cuda()
    dt, As = kevd.symmetric_normalize(Fg, rank)
    ev, U = kevd.symmetric_eig_topk(Fg, rank, dt, As, 16)
    lam0, _ = symmetric_evd(F32.astype(np.float64).T)
    assert np.max(np.abs(ev.cpu().numpy() - lam0[:16]) / lam0[:16]) < 1e-4


@pytest.mark.parametrize("N,pad", [(9001, 5), (12288, 0)])
def test_symmetric_fp32_gram(kevd, N, pad):
    """The one-Gram form of the FP32 Gram kernel: A_s = F^T D~^-1 F from FP32 F
    (FP32 products and split sums, FP64 across splits) against FP64 sums of the
    same FP32 values, F passed as a view with leading dimension N + pad."""
    X, eps, _ = make_config("ks200k", N=N)
    F = arpc(X, eps, 200, 50, 4)["F"]
    F32 = np.ascontiguousarray(F.T, dtype=np.float32)
    rank = F32.shape[0]
    Fe = F32.astype(np.float64).T
    Fbuf = torch.full((rank, N + pad), float("nan"), dtype=torch.float32)
    Fbuf[:, :N] = torch.from_numpy(F32)
    dt, As = kevd.symmetric_normalize(Fbuf.cuda()[:, :N], rank)
    d0 = Fe @ (Fe.T @ np.ones(N))
    assert np.max(np.abs(dt.cpu().numpy() - d0) / d0) < 1e-6
    A0 = Fe.T @ (Fe / d0[:, None])
    As = As.cpu().numpy()
    assert np.array_equal(As, As.T)
    assert np.max(np.abs(As - A0)) < 2e-6 * np.max(np.abs(A0))


def test_constant_eigvec_fix_matches_oracle(kevd):
    rng = np.random.Generator(np.random.PCG64(3))
    N, k = 3000, 20
    U0 = np.linalg.qr(rng.standard_normal((N, k)))[0]
    V0 = constant_eigvec_fix(U0)
    Ug = torch.from_numpy(np.ascontiguousarray(U0.T)).cuda()
    kevd.constant_eigvec_fix(Ug)
    V = Ug.cpu().numpy().T
    assert np.allclose(V[:, 0], 1 / np.sqrt(N), atol=1e-14)
    assert np.max(np.abs(V.T @ V - np.eye(k))) < 1e-13
    s = np.sign(np.sum(V * V0, axis=0))                 # oracle QR may flip column signs
    assert np.max(np.abs(V - V0 * s)) < 1e-12


def test_concurrent_streams_match_sequential(kevd):
    """Normalisation and eigensolves driven by four host threads on their own
    streams (one cuSOLVER/cuBLAS handle per thread) return exactly the results
    of the same calls made in sequence."""
    from concurrent.futures import ThreadPoolExecutor
    cases = []
    for q in range(8):
        X, eps, _ = make_config("ks200k", N=3000 + 500 * q)
        F = arpc(X, eps, 96 + 16 * q, 32, 20 + q)["F"]
        cases.append(torch.from_numpy(np.ascontiguousarray(F.T)).cuda())

    def run(F):
        rk = F.shape[0]
        dt, qt, A, C = kevd.bistoch_normalize(F, rk)
        ev, U, _ = kevd.eig_topk(F, rk, dt, A, C, 8)
        torch.cuda.current_stream().synchronize()
        return ev.cpu(), U.cpu()

    seq = [run(F) for F in cases]
    streams = [torch.cuda.Stream() for _ in range(4)]

    def worker(w):
        out = {}
        with torch.cuda.stream(streams[w]):
            for i in range(w, len(cases), 4):
                out[i] = run(cases[i])
        return out

    par = {}
    with ThreadPoolExecutor(4) as pool:
        for f in [pool.submit(worker, w) for w in range(4)]:
            par.update(f.result())
    for i, (ev, U) in enumerate(seq):
        assert torch.equal(par[i][0], ev) and torch.equal(par[i][1], U)
