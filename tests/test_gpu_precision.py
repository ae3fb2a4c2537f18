"""GPU parity of the precision form (BF16 hi/lo split products on the tensor
cores, FP32 F; FP64 rho, H, reject, L, degrees and eigensolves) against the
FP64 oracle run on the same FP32 inputs (-m gpu).

Tolerances.  The bar for this form is eigenvalues within 1e-4 relative.  For the
factor itself: each split product carries ~2^-16 relative error, which gives
~5e-6 in kernel entries; the forward substitution divides by L_jj, and the
late pivots of these problems have L_jj ~ 0.05, so late columns of F may
differ by up to ~1e-4.  Bars: F 1e-3 absolute, rho 5e-4 absolute, sum(rho)
1e-5 relative.

Pivot sequences.  The split products perturb rho by ~1e-6, so a draw near a
CDF edge may pick a neighbouring pivot and the sequence then leaves the
oracle's.  Every check is therefore made against the replay oracle
(oracle.pchol.pchol_given_pivots): the FP64 factor of the pivot sequence the
GPU accepted.  Where the GPU's proposals equal the oracle's own ARPC run, the
two oracle factors agree too (checked); where they leave it, the first
differing draw must sit within 1e-5 of a CDF or accept edge.  No case skips.
"""
import os

import numpy as np
import pytest
import torch

from datagen import make_config
from oracle.pchol import arpc, greedy_pchol, pchol_given_pivots
from oracle.alg1 import bistochastic_evd
from tests.helpers import compare_eigpairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kevd():
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as m
    return m


def _near(ref, tol=1e-5):
    for rnd, lg in enumerate(ref["log"]):
        if np.min(lg["prop_margin"]) < tol or np.min(np.abs(lg["reject_margin"])) < tol:
            return rnd
    return None


def _blocks(n, m=64):
    """Pivot blocks of m for the replay (any grouping gives the same factor up to rounding)."""
    return [m] * (n // m) + ([n % m] if n % m else [])


def _run(kevd, name, N, r, b, seed, q=None):
    X, eps, cfg = make_config(name, N=N)
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    ref = arpc(X32.astype(np.float64), eps, r, b, seed)
    out = kevd.rpchol_factor(torch.from_numpy(X32).cuda(), eps, r, mode="arpc", b=b, seed=seed,
                             record_proposals=True)
    return X32, eps, ref, out


def _replay(X32, eps, out):
    """FP64 factor of the GPU's accepted pivots, and those pivots."""
    S = out["pivots"].cpu().numpy()[: out["rank"]]
    return pchol_given_pivots(X32.astype(np.float64), eps, S, blocks=_blocks(len(S))), S


def _same_or_near_edge(ref, out):
    """True if the GPU's proposals equal the oracle's ARPC; else the first differing round
    must be one with a draw within 1e-5 of a CDF or accept edge."""
    props = out["proposals"].cpu().numpy()
    for rnd, lg in enumerate(ref["log"]):
        if rnd >= len(props) or props[rnd].tolist() != lg["proposals"].tolist():
            near = _near({"log": ref["log"][rnd:rnd + 1]})
            assert near is not None, "round %d differs with every oracle margin above 1e-5" % rnd
            return False
    return out["rank"] == ref["F"].shape[1]


@pytest.mark.parametrize("name,N,r,b,seed", [
    ("ks200k", 5000, 256, 64, 1003),      # BN = 64
    ("vsa524k", 1037, 100, 24, 5),        # BN = 32, d = 96 (padded K chunk), ragged N
    ("vsa2m", 4000, 256, 128, 9),         # BN = 128, d = 128
])
def test_bf16x3_factor_matches_oracle(kevd, name, N, r, b, seed):
    X32, eps, ref, out = _run(kevd, name, N, r, b, seed)
    assert out["F"].dtype == torch.float32
    rp, S = _replay(X32, eps, out)
    if _same_or_near_edge(ref, out):
        assert S.tolist() == ref["pivots"].tolist()
        assert np.max(np.abs(rp["F"] - ref["F"])) < 1e-12
    F = out["F"].cpu().numpy().astype(np.float64).T[:, : out["rank"]]
    assert np.max(np.abs(F - rp["F"])) < 1e-3
    assert np.max(np.abs(F[:, :8] - rp["F"][:, :8])) < 5e-5          # first block: no amplification
    rho = out["rho"].cpu().numpy()
    assert np.max(np.abs(rho - rp["rho"])) < 5e-4
    assert abs(out["trace_err"] - rp["rho"].sum()) / rp["rho"].sum() < 1e-5


def test_bf16x3_greedy_matches_oracle(kevd):
    """Greedy in FP32: F equals the FP64 factor of the GPU's own pivot sequence, and
    every pivot is a valid argmax: its FP64 residual is within 1e-5 of the largest
    (argmax near-ties may resolve either way under FP32 rounding)."""
    X, eps, _ = make_config("ks2k", N=1200)
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    F0, S0, rho0, _ = greedy_pchol(X32.astype(np.float64), eps, 48)
    out = kevd.rpchol_factor(torch.from_numpy(X32).cuda(), eps, 48, mode="greedy")
    S = out["pivots"].cpu().numpy()[: out["rank"]]
    rp = pchol_given_pivots(X32.astype(np.float64), eps, S)
    F = out["F"].cpu().numpy().astype(np.float64).T[:, : out["rank"]]
    assert np.max(np.abs(F - rp["F"])) < 1e-3
    Fp = rp["F"]
    for j, s in enumerate(S):
        res = 1.0 - np.sum(Fp[:, :j] ** 2, axis=1)          # FP64 residual diagonal before pivot j
        assert res[s] >= res.max() - 1e-5, (j, res[s], res.max())
    n_eq = next((i for i, (a, c) in enumerate(zip(S, S0)) if a != c), len(S0))
    assert n_eq >= 16, n_eq                                  # the sequences agree at least this long


def _precision_pipeline(kevd, out, k, strict=False):
    """Normalisation and top-k of the precision form; strict: the subspace top-k must
    take and pass its residual check (an error instead of the subset-solver fallback)."""
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], out["rank"])
    if strict:
        os.environ["KEVD_TOPK"] = "subspace"
    try:
        ev, U, kept = kevd.eig_topk(out["F"], out["rank"], dt, A, C, k, tau=1e-6)
    finally:
        os.environ.pop("KEVD_TOPK", None)
    return ev.cpu().numpy(), U.cpu().numpy().T


def _check_eigenvectors(ev, U, lam0, U0, gap=1e-2, tol=1e-4):
    """Eigenvectors of the precision form (the FP32 lift on the tensor cores) against the
    oracle's on the replayed FP64 factor: each column whose eigenvalue lies at least `gap`
    from its neighbours (the lifted vector's perturbation is ~ |dP| / gap) within `tol` of
    its largest entry after sign alignment; every cluster's subspace within 1e-2 radians."""
    from tests.helpers import max_angle, clusters
    k = len(lam0)
    worst = 0.0
    checked = 0
    for j in range(k):
        g = min([abs(lam0[j] - lam0[i]) for i in (j - 1, j + 1) if 0 <= i < k] + [np.inf])
        if g < gap:
            continue
        u0 = U0[:, j]
        u = U[:, j] * np.sign(np.dot(U[:, j], u0))
        err = np.max(np.abs(u - u0)) / np.max(np.abs(u0))
        worst = max(worst, err)
        checked += 1
        assert err < tol, (j, lam0[j], g, err)
    for c in clusters(lam0, 1e-6):
        assert max_angle(U0[:, c], U[:, c]) < 1e-2
    print("eigenvectors: %d separated columns, worst %.2e of the column maximum" % (checked, worst))
    assert checked >= 1


def _rescored_trace(out, N):
    """sum(rho) of the returned FP32 factor recomputed in FP64: tr(K - F F^T) = sum_i (1 - |F_i|^2)."""
    F = out["F"].cpu().numpy().astype(np.float64)[: out["rank"]]
    return float(np.sum(np.maximum(1.0 - np.sum(F * F, axis=0), 0.0)))


def test_bf16x3_pipeline_eigenvalues(kevd):
    """Precision form end to end against the FP64 oracle (Algorithm 1 by Householder
    QR on the FP64 factor of the same pivots): top-32 eigenvalues within 1e-4
    relative, and the trace-norm error of the returned factor, re-scored in FP64,
    within 1e-4 relative of the FP64 factor's."""
    X32, eps, ref, out = _run(kevd, "ks200k", 6000, 256, 64, 1004)
    rp, S = _replay(X32, eps, out)
    if _same_or_near_edge(ref, out):
        assert np.max(np.abs(rp["F"] - ref["F"])) < 1e-12
    k = 32
    ev, U = _precision_pipeline(kevd, out, k)
    lam0, U0 = bistochastic_evd(rp["F"], k)
    erel = np.max(np.abs(ev - lam0) / np.abs(lam0))
    assert erel < 1e-4, erel
    assert abs(ev[0] - 1.0) < 1e-4
    _check_eigenvectors(ev, U, lam0, U0)
    tr64 = _rescored_trace(out, 6000)
    assert abs(tr64 - rp["rho"].sum()) / rp["rho"].sum() < 1e-4, (tr64, rp["rho"].sum())


@pytest.mark.slow
def test_bf16x3_pipeline_eigenvalues_large(kevd):
    """The same end-to-end check at N = 131,072 points of the vsa2m workload (d = 128,
    b = 128, r = 2,048; rank above 1,500, where 1/L_jj amplification is largest):
    top-64 eigenvalues within 1e-4 relative of the FP64 oracle on the replayed factor,
    through the subspace top-k in strict mode (b = 160 <= rank / 3: no fallback)."""
    X, eps, cfg = make_config("vsa2m", N=131072)
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    out = kevd.rpchol_factor(torch.from_numpy(X32).cuda(), eps, 2048, mode="arpc", b=128, seed=1005)
    assert out["rank"] >= 1500, out["rank"]
    rp, S = _replay(X32, eps, out)
    F = out["F"].cpu().numpy().astype(np.float64).T[:, : out["rank"]]
    ferr = np.max(np.abs(F - rp["F"]))
    k = 64
    ev, U = _precision_pipeline(kevd, out, k, strict=True)
    del F
    lam0, U0 = bistochastic_evd(rp["F"], k)
    erel = np.max(np.abs(ev - lam0) / np.abs(lam0))
    tr64 = _rescored_trace(out, X.shape[0])
    print("rank %d, max|F - F64| %.3e, eig rel %.3e, trace %.6e vs %.6e" % (out["rank"], ferr, erel, tr64,
                                                                              rp["rho"].sum()))
    assert ferr < 1e-3, ferr
    assert erel < 1e-4, erel
    assert abs(tr64 - rp["rho"].sum()) / rp["rho"].sum() < 1e-3, (tr64, rp["rho"].sum())
    _check_eigenvectors(ev, U, lam0, U0)


def test_bf16x3_rejects_wrong_dtypes(kevd):
    X = torch.zeros((100, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(kevd.KevdError):
        kevd.rpchol_factor(X, 1.0, 16, precision="bf16x3")


# (N, rank, pad): pad > 0 passes F as a view with leading dimension N + pad;
# N = 3001, 777 and odd pads take the 4-byte copy path, the rest 16-byte copies;
# ranks 128 / 129 / 300 end exactly on, one past and inside a 128-column tile.
# pad: F is a view with leading dimension N + pad.  ldf = N + pad a multiple of 4
# (and F 16-byte aligned) takes the tensor-core Gram (TMA-staged tiles, exact
# leading slice product); other ldf the FFMA Gram.  N = 20,037 and 300,000
# end in a partial 64-row stage; rank 129 / 300 / 1,000 leave ragged tiles.
@pytest.mark.parametrize("N,rank,pad,gram", [(3001, 200, 0, None), (20000, 300, 0, None), (777, 64, 0, None),
                                             (8192, 128, 0, None), (8192, 129, 4, None), (5000, 260, 3, None),
                                             (40000, 140, 0, None), (20037, 300, 3, None), (20000, 300, 0, "ffma"),
                                             (60000, 1000, 0, None)])
def test_bf16x3_normalize_matches_fp64(kevd, monkeypatch, N, rank, pad, gram):
    """Degree vectors (FP32 products, FP64 block sums) and Grams of an FP32 F
    against the same quantities in FP64 from the same FP32 values; the diagonal
    of each Gram carries no accumulation bias (mean signed relative error)."""
    from oracle.alg1 import degree_vectors
    if gram:
        monkeypatch.setenv("KEVD_GRAM", gram)
    X, eps, _ = make_config("ks200k" if rank < 500 else "vsa2m", N=N)
    F64 = arpc(X, eps, rank, 16 if rank < 500 else 100, 3)["F"]
    F32 = np.ascontiguousarray(F64.T, dtype=np.float32)            # (rank', N) = column-major N x rank'
    Fe = F32.astype(np.float64).T
    rk = Fe.shape[1]
    Fbuf = torch.full((rk, N + pad), float("nan"), dtype=torch.float32)
    Fbuf[:, :N] = torch.from_numpy(F32)
    Fg = Fbuf.cuda()[:, :N]
    dt, qt, A, C = kevd.bistoch_normalize(Fg, rk)
    d0, q0 = degree_vectors(Fe)
    assert np.max(np.abs(dt.cpu().numpy() - d0) / d0) < 1e-6
    assert np.max(np.abs(qt.cpu().numpy() - q0) / q0) < 1e-6
    A0 = Fe.T @ (Fe / (d0 * d0)[:, None])
    C0 = Fe.T @ (Fe / q0[:, None])
    A = A.cpu().numpy()
    C = C.cpu().numpy()
    assert np.array_equal(A, A.T) and np.array_equal(C, C.T)
    # FP32 products (FFMA), or hi/mid slice products with the leading one summed
    # exactly (tensor cores): ~1e-7 relative
    assert np.max(np.abs(A - A0)) < 2e-6 * np.max(np.abs(A0))
    assert np.max(np.abs(C - C0)) < 2e-6 * np.max(np.abs(C0))
    # no systematic bias: truncating accumulation would pull every diagonal entry
    # down by ~1e-5 relative; round-to-nearest sums leave a mean of ~1e-7 at most
    for G, G0 in ((A, A0), (C, C0)):
        bias = np.mean((np.diag(G) - np.diag(G0)) / np.diag(G0))
        assert abs(bias) < 1e-6, bias


@pytest.mark.slow
def test_bf16x3_normalize_matches_fp64_300k(kevd):
    """The same check at N = 300,000 rows of the vsa2m workload (d = 128), a factor of
    rank ~700 in FP32: many row splits and whole-wave grids of the tensor-core Gram."""
    from oracle.alg1 import degree_vectors
    X, eps, _ = make_config("vsa2m", N=300000)
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    out = kevd.rpchol_factor(torch.from_numpy(X32).cuda(), eps, 768, mode="arpc", b=128, seed=11)
    rk = out["rank"]
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], rk)
    Fe = out["F"][:rk].double().cpu().numpy().T
    d0, q0 = degree_vectors(Fe)
    A0 = Fe.T @ (Fe / (d0 * d0)[:, None])
    C0 = Fe.T @ (Fe / q0[:, None])
    A = A.cpu().numpy()
    C = C.cpu().numpy()
    assert np.max(np.abs(dt.cpu().numpy() - d0) / d0) < 1e-6
    assert np.max(np.abs(A - A0)) < 2e-6 * np.max(np.abs(A0))
    assert np.max(np.abs(C - C0)) < 2e-6 * np.max(np.abs(C0))
    for G, G0 in ((A, A0), (C, C0)):
        assert abs(np.mean((np.diag(G) - np.diag(G0)) / np.diag(G0))) < 1e-6


# (N, rank, k, pad): odd N takes the 4-byte copy path and scalar FP64 stores,
# pad > 0 passes F as a view with leading dimension N + pad; k = 40 / 130
# leave a ragged 128-wide output tile, rank = 201 a ragged 16-column chunk.
@pytest.mark.parametrize("N,rank,k,pad", [(5001, 201, 40, 0), (8192, 256, 130, 4), (12000, 160, 16, 3)])
def test_fp32_lift_matches_fp64_lift(kevd, N, rank, k, pad):
    """eig_topk with FP32 F against eig_topk with the same values in FP64 F and the
    same d~, A, C: the r x r stage is identical, so U differs only by the lift's FP32
    products and sums (about 1e-7 relative per entry, times the growth of Y)."""
    X, eps, _ = make_config("ks200k", N=N)
    F64 = arpc(X, eps, rank, 16, 5)["F"]
    F32 = np.ascontiguousarray(F64.T, dtype=np.float32)
    rk = F32.shape[0]
    k = min(k, rk)
    Fe = torch.from_numpy(F32.astype(np.float64)).cuda()
    dt, qt, A, C = kevd.bistoch_normalize(Fe, rk)
    ev64, U64, _ = kevd.eig_topk(Fe, rk, dt, A, C, k)
    Fbuf = torch.full((rk, N + pad), float("nan"), dtype=torch.float32)
    Fbuf[:, :N] = torch.from_numpy(F32)
    os.environ["KEVD_TOPK"] = "full"   # the same r x r solver as the FP64 call
    try:
        ev32, U32, _ = kevd.eig_topk(Fbuf.cuda()[:, :N], rk, dt, A, C, k)
    finally:
        os.environ.pop("KEVD_TOPK", None)
    assert torch.equal(ev32, ev64)
    U32 = U32.cpu().numpy()
    U64 = U64.cpu().numpy()
    assert np.all(np.isfinite(U32))
    U32 = U32 * np.sign(np.sum(U32 * U64, axis=1, keepdims=True))   # sign rule ties may differ
    scale = np.max(np.abs(U64), axis=1, keepdims=True)
    assert np.max(np.abs(U32 - U64) / scale) < 1e-4


def _topk(kevd, F, rk, dt, A, C, k, full):
    """full: the subset eigensolver; otherwise the subspace solver, whose failed
    residual check is then an error (no silent fallback)."""
    os.environ["KEVD_TOPK"] = "full" if full else "subspace"
    try:
        ev, U, _ = kevd.eig_topk(F, rk, dt, A, C, k)
    finally:
        os.environ.pop("KEVD_TOPK", None)
    return ev.cpu().numpy(), U.cpu().numpy().T


@pytest.mark.parametrize("N,r,b,k", [(6000, 400, 64, 32), (20000, 700, 100, 64), (30000, 1200, 100, 128)])
def test_subspace_topk_matches_full(kevd, N, r, b, k):
    """Precision form: the FP64 subspace top-k of M (residual-checked Rayleigh-Ritz)
    against the full subset eigensolver on the same d~, A, C: eigenvalues to 1e-6
    relative (the residual bound it enforces); eigenvectors, grouped into clusters of
    relative gap < 1e-2, to 1e-3 after the FP32 lift (residual / gap plus lift noise).
    The subspace call runs in strict mode, so a failed check fails the test."""
    X, eps, _ = make_config("vsa524k", N=N)
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    out = kevd.rpchol_factor(torch.from_numpy(X32).cuda(), eps, r, mode="arpc", b=b, seed=5, precision="bf16x3")
    rk = out["rank"]
    k = max(1, min(k, rk // 6 - 16))   # the subspace path needs 2k + 32 <= rank / 3
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], rk)
    ev_s, U_s = _topk(kevd, out["F"], rk, dt, A, C, k, full=False)
    ev_fa, U_fa = _topk(kevd, out["F"], rk, dt, A, C, k + 1, full=True)
    ev_f, U_f = ev_fa[:k], U_fa[:, :k]
    erel, ang = compare_eigpairs(ev_f, U_f, ev_s, U_s, rel_gap=1e-2, lam_full=ev_fa)
    assert erel < 1e-6, erel
    assert ang < 1e-3, ang


def test_subspace_falls_back_on_flat_spectrum(kevd):
    """A nearly flat spectrum (0.9 .. 1) defeats six power steps; the residual check
    must reject the Ritz pairs (an error in strict mode) and the default call's
    fallback, the subset eigensolver, must give the exact values.
    Route: F = I, d~ = 1, A = I, so M = C = Q diag(lambda) Q^T."""
    n, k = 600, 40   # b = 112 <= n / 3
    rng = np.random.Generator(np.random.PCG64(3))
    lam = np.sort(rng.uniform(0.9, 1.0, n))[::-1].copy()
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Cm = (Q * lam) @ Q.T
    Cm = 0.5 * (Cm + Cm.T)
    I32 = torch.eye(n, dtype=torch.float32).cuda()
    I64 = torch.eye(n, dtype=torch.float64).cuda()
    dt = torch.ones(n, dtype=torch.float64).cuda()
    Cd = torch.from_numpy(np.ascontiguousarray(Cm.T)).cuda()
    with pytest.raises(kevd.KevdError) as ei:
        _topk(kevd, I32, n, dt, I64, Cd, k, full=False)
    from paper_2510_26574_gb300.kevd import KEVD_EEIG
    assert ei.value.status == KEVD_EEIG
    ev, U, _ = kevd.eig_topk(I32, n, dt, I64, Cd, k)
    ev, U = ev.cpu().numpy(), U.cpu().numpy().T
    assert np.max(np.abs(ev - lam[:k]) / lam[:k]) < 1e-10
    assert np.max(np.abs(Cm @ U - U * ev)) < 1e-6


@pytest.mark.slow
def test_subspace_topk_vsa2m_without_fallback(kevd):
    """The vsa2m workload at full size (N = 2,000,000, d = 128, r = 2,048, b = 128,
    k = 256; inner matrix r ~ 1,850 whose top-256 eigenvalues span 1 .. 2e-7): the
    precision form's subspace solver (b = 544) passes its residual check with no
    fallback (strict mode) and matches the subset eigensolver on the same d~, A, C:
    eigenvalues to 1e-6 relative, clusters of relative gap < 1e-2 to 1e-3 radians."""
    X, eps, cfg = make_config("vsa2m")
    Xg = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    del X
    out = kevd.rpchol_factor(Xg, eps, cfg["r"], mode="arpc", b=cfg["b"], seed=1005)
    del Xg
    rk, k = out["rank"], cfg["k"]
    assert 2 * k + 32 <= rk // 3, rk
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], rk)
    ev_s, U_s = _topk(kevd, out["F"], rk, dt, A, C, k, full=False)
    ev_fa, U_fa = _topk(kevd, out["F"], rk, dt, A, C, k + 1, full=True)
    erel, ang = compare_eigpairs(ev_fa[:k], U_fa[:, :k], ev_s, U_s, rel_gap=1e-2, lam_full=ev_fa)
    print("rank %d, lambda_k %.3e, eig rel %.2e, max cluster angle %.2e" % (rk, ev_s[-1], erel, ang))
    assert erel < 1e-6, erel
    assert ang < 1e-3, ang
