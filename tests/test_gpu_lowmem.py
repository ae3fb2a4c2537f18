"""GPU parity of the low-memory form (Appendix A, closing paragraph; Remark of
Section 4.2) through the C-ABI (-m gpu).  rpchol_factor_lowmem keeps only the
pivots S and W = F(S,:); bistoch_normalize_lowmem and eig_topk_lowmem rebuild
what they need of F = K(:,S) W^-T panel by panel.

* Against the oracle (oracle/lowmem.py, pinned to ARPC, to the Cholesky factor
  of K(S,S) and to the dense P): identical proposals, pivots and rounds (a
  difference is only tolerated at a near-edge draw; W and rho are then checked
  against the replay oracle's FP64 factor of the GPU's own pivots), W and
  rho to 1e-10; d~ and q~ to 1e-12 and A, C to 1e-10 relative; eigenpairs at
  the FP64 bars (eigenvalues 1e-10 relative, cluster subspace angle 1e-8).
* Greedy pivoting against the greedy oracle.
* Against the stored-F path on the same inputs: same pivots, W = F(S,:).
* Small panels (KEVD_LOWMEM_PANEL) so that N spans many panels and a ragged one.
* An out-of-range pivot is reported as KEVD_EINVAL (checked before any read).
* Full size (ks200k: N = 200,000, d = 64, r = 1,024, b = 64): the pivots of the
  stored-F path, W = F(S,:) and rho to 1e-10, d~ and the top-64 eigenvalues of
  the stored-F path.
"""
import numpy as np
import pytest
import torch

from datagen import make_config
from oracle.pchol import greedy_pchol, pchol_given_pivots
from oracle.lowmem import arpc_lowmem, lowmem_rows, normalize_lowmem
from oracle.alg1 import bistochastic_evd
from tests.helpers import compare_eigpairs, first_divergence

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kevd():
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as m
    return m


def _gpu(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def _near_edge(log, rnd, tol=1e-9):
    lg = log[rnd]
    return bool(np.min(lg["prop_margin"]) < tol or np.min(np.abs(lg["reject_margin"])) < tol)


def _check_rounds(out, ref):
    """True if every round's proposals equal the oracle's.  A difference is only
    allowed at a draw within 1e-9 of a CDF or accept edge (then False: the caller
    checks against the replay of the GPU's own pivots instead)."""
    props = out["proposals"].cpu().numpy()
    for rnd, lg in enumerate(ref["log"]):
        if rnd >= len(props) or props[rnd].tolist() != lg["proposals"].tolist():
            assert _near_edge(ref["log"], rnd), "round %d proposals differ away from a CDF edge" % rnd
            return False
    assert out["rounds"] == ref["rounds"] == len(ref["log"])
    return True


@pytest.mark.parametrize("N,r,b,seed,panel", [(3000, 128, 32, 11, None), (5000, 256, 32, 1002, "256"),
                                              (1037, 100, 24, 7, "64")])
def test_factor_matches_oracle(kevd, monkeypatch, N, r, b, seed, panel):
    if panel:
        monkeypatch.setenv("KEVD_LOWMEM_PANEL", panel)
    X, eps, _ = make_config("ks200k", N=N)
    ref = arpc_lowmem(X, eps, r, b, seed)
    out = kevd.rpchol_factor_lowmem(_gpu(X), eps, r, b=b, seed=seed, record_proposals=True)
    same = _check_rounds(out, ref)
    rk = out["rank"]
    S = out["pivots"].cpu().numpy()[:rk]
    if same:
        assert rk == len(ref["pivots"])
        i = first_divergence(S, ref["pivots"])
        assert i is None, "pivot %d differs" % i
        Wref, rho_ref = ref["W"], ref["rho"]
    else:
        rp = pchol_given_pivots(X, eps, S, blocks=[16] * (rk // 16) + [rk % 16] * (rk % 16 > 0))
        Wref, rho_ref = rp["F"][S], rp["rho"]
        ref = dict(ref, rho=rho_ref)
    W = out["W"].cpu().numpy()
    assert np.max(np.abs(W[:rk, :rk] - Wref)) < 1e-10
    assert np.all(np.triu(W, 1) == 0)
    assert np.all(W[rk:, :] == 0) and np.all(W[:, rk:] == 0)
    rho = out["rho"].cpu().numpy()
    assert np.max(np.abs(rho - ref["rho"])) < 1e-10
    assert abs(out["trace_err"] - ref["rho"].sum()) <= 1e-10 * N


def test_greedy_matches_oracle(kevd, monkeypatch):
    monkeypatch.setenv("KEVD_LOWMEM_PANEL", "320")
    X, eps, _ = make_config("ks2k")
    F0, S0, rho0, _ = greedy_pchol(X, eps, 96)
    out = kevd.rpchol_factor_lowmem(_gpu(X), eps, 96, mode="greedy")
    assert out["rank"] == len(S0) == 96
    assert out["pivots"].cpu().numpy().tolist() == S0.tolist()
    W = out["W"].cpu().numpy()
    assert np.max(np.abs(W - F0[S0])) < 1e-12
    assert np.max(np.abs(out["rho"].cpu().numpy() - rho0)) < 1e-12


@pytest.mark.parametrize("panel", [None, "4096"])
def test_factor_matches_stored_F_path(kevd, monkeypatch, panel):
    if panel:
        monkeypatch.setenv("KEVD_LOWMEM_PANEL", panel)
    X, eps, _ = make_config("ks200k", N=20000)
    Xg = _gpu(X)
    ref = kevd.rpchol_factor(Xg, eps, 512, mode="arpc", b=64, seed=3)
    out = kevd.rpchol_factor_lowmem(Xg, eps, 512, b=64, seed=3)
    rk = out["rank"]
    assert rk == ref["rank"] and out["rounds"] == ref["rounds"]
    S = out["pivots"].cpu().numpy()[:rk]
    assert S.tolist() == ref["pivots"].cpu().numpy()[:rk].tolist()
    F = ref["F"].cpu().numpy().T[:, :rk]
    W = out["W"].cpu().numpy()[:rk, :rk]
    assert np.max(np.abs(W - F[S])) < 1e-10
    assert np.max(np.abs(out["rho"].cpu().numpy() - ref["rho"].cpu().numpy())) < 1e-10


@pytest.mark.parametrize("panel", [None, "192"])
def test_normalize_and_eig_match_oracle(kevd, monkeypatch, panel):
    if panel:
        monkeypatch.setenv("KEVD_LOWMEM_PANEL", panel)
    N, r, b, seed, k = 3000, 200, 40, 5, 24
    X, eps, _ = make_config("ks200k", N=N)
    ref = arpc_lowmem(X, eps, r, b, seed)
    Xg = _gpu(X)
    out = kevd.rpchol_factor_lowmem(Xg, eps, r, b=b, seed=seed)
    rk = out["rank"]
    assert out["pivots"].cpu().numpy()[:rk].tolist() == ref["pivots"].tolist()
    S, W = ref["pivots"], ref["W"]
    dt0, qt0, A0, C0 = normalize_lowmem(X, eps, S, W)
    dt, qt, A, C = kevd.bistoch_normalize_lowmem(Xg, eps, out["pivots"], out["W"], rk)
    dt, qt, A, C = (t.cpu().numpy() for t in (dt, qt, A, C))
    assert np.max(np.abs(dt - dt0) / dt0) < 1e-12
    assert np.max(np.abs(qt - qt0) / qt0) < 1e-12
    assert np.max(np.abs(A - A0)) < 1e-10 * np.max(np.abs(A0))
    assert np.max(np.abs(C - C0)) < 1e-10 * np.max(np.abs(C0))
    assert np.all(A == A.T) and np.all(C == C.T)
    lam0, U0 = bistochastic_evd(lowmem_rows(X, eps, S, W, np.arange(N)))
    ev, U, kept = kevd.eig_topk_lowmem(Xg, eps, out["pivots"], out["W"], rk, *(torch.from_numpy(a).cuda() for a in
                                                                             (dt, A, C)), k)
    ev, U = ev.cpu().numpy(), U.cpu().numpy().T
    assert np.all(np.diff(ev) <= 0)
    erel, ang = compare_eigpairs(lam0[:k], U0[:, :k], ev, U, lam_full=lam0)
    assert erel < 1e-10 and ang < 1e-8, (erel, ang)
    assert np.max(np.abs(U.T @ U - np.eye(k))) < 1e-10


def test_out_of_range_pivot_is_an_error(kevd):
    X, eps, _ = make_config("ks200k", N=1000)
    Xg = _gpu(X)
    out = kevd.rpchol_factor_lowmem(Xg, eps, 64, b=32, seed=1)
    rk = out["rank"]
    bad = out["pivots"].clone()
    bad[rk // 2] = 1000                      # == N
    with pytest.raises(kevd.KevdError) as e:
        kevd.bistoch_normalize_lowmem(Xg, eps, bad, out["W"], rk)
    assert e.value.status == 1
    dt, qt, A, C = kevd.bistoch_normalize_lowmem(Xg, eps, out["pivots"], out["W"], rk)
    bad[rk // 2] = -1
    with pytest.raises(kevd.KevdError) as e:
        kevd.eig_topk_lowmem(Xg, eps, bad, out["W"], rk, dt, A, C, 4)
    assert e.value.status == 1


def test_fullsize_ks200k_matches_stored_F_path(kevd):
    X, eps, _ = make_config("ks200k")
    N = X.shape[0]
    Xg = _gpu(X)
    ref = kevd.rpchol_factor(Xg, eps, 1024, mode="arpc", b=64, seed=0)
    out = kevd.rpchol_factor_lowmem(Xg, eps, 1024, b=64, seed=0)
    rk = out["rank"]
    assert rk == ref["rank"]
    S = out["pivots"][:rk]
    assert torch.equal(S, ref["pivots"][:rk])
    Fs = ref["F"][:rk, S].T                                   # F(S,:) from the stored factor
    assert torch.max(torch.abs(out["W"][:rk, :rk] - Fs)).item() < 1e-10
    assert torch.max(torch.abs(out["rho"] - ref["rho"])).item() < 1e-10
    dt_f, qt_f, A_f, C_f = kevd.bistoch_normalize(ref["F"][:rk], rk)
    ev_f, _, _ = kevd.eig_topk(ref["F"][:rk], rk, dt_f, A_f, C_f, 64)
    del ref, Fs
    dt, qt, A, C = kevd.bistoch_normalize_lowmem(Xg, eps, out["pivots"], out["W"], rk)
    assert torch.max(torch.abs(dt - dt_f) / dt_f).item() < 1e-12
    assert torch.max(torch.abs(qt - qt_f) / qt_f).item() < 1e-12
    ev, U, _ = kevd.eig_topk_lowmem(Xg, eps, out["pivots"], out["W"], rk, dt, A, C, 64)
    assert torch.max(torch.abs(ev - ev_f) / ev_f.abs()).item() < 1e-10
    assert U.shape == (64, N)
