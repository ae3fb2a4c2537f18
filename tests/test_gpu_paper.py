"""The paper-shaped workloads of Section 4 on the GPU (-m gpu).

* paper32k (Section 4.1's set-up: the paper's initial condition, J = 64 delays at one
  grid point, eps = 32 J): the FP64 path against the FP64 factor of the same pivots, and
  the precision form's normalisation and eigensolve against the spectrum of its own
  factor (the FP32 factor itself is at its resolution limit on this wide kernel).
* paper131k (Section 4.2's set-up, median-rule eps) at one rank of the paper's sweep
  (r = 512): the FP64 path against the complete oracle (Algorithm 2 + Algorithm 1 by
  Householder QR) at the FP64 tolerances, and the precision form against the replay.
"""
import numpy as np
import pytest
import torch

from datagen import make_config
from oracle.alg1 import bistochastic_evd
from oracle.pchol import arpc, pchol_given_pivots
from tests.helpers import compare_eigpairs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def kevd():
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as m
    return m


def _blocks(n, b=64):
    return [b] * (n // b) + [n % b] * (n % b > 0)


def _precision_vs_replay(kevd, X, eps, r, b, k, seed, tol=None):
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    out = kevd.rpchol_factor(torch.from_numpy(X32).cuda(), eps, r, mode="arpc", b=b, seed=seed, tol=tol)
    rank = out["rank"]
    S = out["pivots"].cpu().numpy()[:rank]
    rp = pchol_given_pivots(X32.astype(np.float64), eps, S, blocks=_blocks(rank))
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], rank)
    ev, U, kept = kevd.eig_topk(out["F"], rank, dt, A, C, k, tau=1e-6)
    lam0, _ = bistochastic_evd(rp["F"], k)
    ev = ev.cpu().numpy()
    # the 1e-4 relative bar on the eigenvalues above 1e-4 (P~'s leading eigenvalue is 1);
    # below, the spectrum of a wide kernel reaches the factor's FP32 noise, bounded in absolute terms
    big = np.abs(lam0) >= 1e-4
    erel = np.max(np.abs(ev[big] - lam0[big]) / np.abs(lam0[big]))
    eabs = np.max(np.abs(ev[~big] - lam0[~big])) if (~big).any() else 0.0
    print("eigenvalues: %d of %d above 1e-4, smallest %.3e / %.3e; abs err below %.3e" %
          (big.sum(), k, lam0[-1], ev[-1], eabs))
    assert eabs < 1e-5, eabs
    F = out["F"].cpu().numpy().astype(np.float64).T[:, :rank]
    tr64 = float(np.sum(np.maximum(1.0 - np.sum(F * F, axis=1), 0.0)))   # tr(K - F F^T), re-scored in FP64
    trel = abs(tr64 - rp["rho"].sum()) / rp["rho"].sum()
    print("rank %d, max|F - F64| %.3e, eig rel %.3e, trace rel %.3e" % (rank, np.max(np.abs(F - rp["F"])), erel,
                                                                          trel))
    return rank, np.max(np.abs(F - rp["F"])), erel, trel


def test_paper32k_precision_pipeline_and_fp32_limit(kevd):
    """paper32k in the precision form.  With eps = 32 J the kernel is close to 1 for most
    pairs and the residuals K - F F^T cancel below FP32's resolution: the FP32 factor's own
    spectrum differs from the FP64 factor of the same pivots by up to ~1 % (measured
    0.9 % at rank 167), the precision form's accuracy limit on this workload (the paper's
    FP32 run reports an 8.91 % trace-norm error).  What the GPU stages after the factor
    must do holds: normalisation and the top-k eigensolve reproduce the FP64 spectrum of
    the returned factor (1e-5 relative on the eigenvalues above 1e-4)."""
    X, eps, cfg = make_config("paper32k")
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    out = kevd.rpchol_factor(torch.from_numpy(X32).cuda(), eps, cfg["r"], mode="arpc", b=cfg["b"], seed=1006,
                             tol=1e-4)
    rank, k = out["rank"], cfg["k"]
    assert 64 < rank < cfg["r"], rank
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], rank)
    ev, U, kept = kevd.eig_topk(out["F"], rank, dt, A, C, k, tau=1e-6)
    ev = ev.cpu().numpy()
    F = out["F"].cpu().numpy().astype(np.float64).T[:, :rank]
    lamF, _ = bistochastic_evd(F, k)
    big = np.abs(lamF) >= 1e-4
    rel = np.max(np.abs(ev[big] - lamF[big]) / np.abs(lamF[big]))
    print("paper32k: rank %d, %d eigenvalues above 1e-4, pipeline vs its factor %.3e" % (rank, big.sum(), rel))
    assert rel < 1e-5, rel
    assert abs(ev[0] - 1.0) < 1e-5


def test_paper32k_fp64_against_oracle(kevd):
    """paper32k on the FP64 path (r = 256, below the kernel's numerical rank) against the
    complete oracle: the eigenvalues above 1e-4 within 1e-8 relative, the rest within 1e-10
    absolute, and the trace-norm error within 1e-8 relative (F itself is ill-determined:
    cond K(S,S) is large for this wide kernel)."""
    X, eps, cfg = make_config("paper32k")
    X = X.astype(np.float64)
    r, b, k, seed = 256, cfg["b"], cfg["k"], 1006
    out = kevd.rpchol_factor(torch.from_numpy(X).cuda(), eps, r, mode="arpc", b=b, seed=seed)
    rank = out["rank"]
    S = out["pivots"].cpu().numpy()[:rank]
    rp = pchol_given_pivots(X, eps, S, blocks=_blocks(rank))
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], rank)
    ev, U, kept = kevd.eig_topk(out["F"], rank, dt, A, C, k)
    ev = ev.cpu().numpy()
    lam0, _ = bistochastic_evd(rp["F"], k)
    big = np.abs(lam0) >= 1e-4
    erel = np.max(np.abs(ev[big] - lam0[big]) / np.abs(lam0[big]))
    eabs = np.max(np.abs(ev[~big] - lam0[~big])) if (~big).any() else 0.0
    trel = abs(out["trace_err"] - rp["rho"].sum()) / rp["rho"].sum()
    print("paper32k FP64: rank %d, eig rel %.3e (above 1e-4), abs %.3e below, trace rel %.3e" % (rank, erel, eabs,
                                                                                                trel))
    assert erel < 1e-8, erel
    assert eabs < 1e-10, eabs
    assert trel < 1e-8, trel


def test_paper131k_fp64_full_oracle(kevd):
    X, eps, cfg = make_config("paper131k")
    X = X.astype(np.float64)
    r, b, k, seed = 512, cfg["b"], cfg["k"], 1007
    out = kevd.rpchol_factor(torch.from_numpy(X).cuda(), eps, r, mode="arpc", b=b, seed=seed,
                             record_proposals=True)
    ref = arpc(X, eps, r, b, seed)
    rank = out["rank"]
    S = out["pivots"].cpu().numpy()[:rank]
    props = out["proposals"].cpu().numpy()
    for rnd, lg in enumerate(ref["log"]):
        if rnd >= len(props) or props[rnd].tolist() != lg["proposals"].tolist():
            near = np.min(lg["prop_margin"]) < 1e-9 or np.min(np.abs(lg["reject_margin"])) < 1e-9
            assert near, "round %d differs away from a CDF edge" % rnd
            ref = pchol_given_pivots(X, eps, S, blocks=_blocks(rank))
            ref["pivots"] = S
            break
    assert rank == ref["F"].shape[1]
    assert S.tolist() == ref["pivots"].tolist()
    F = out["F"].cpu().numpy().T[:, :rank]
    assert np.max(np.abs(F - ref["F"])) < 1e-10
    dt, qt, A, C = kevd.bistoch_normalize(out["F"], rank)
    ev, U, kept = kevd.eig_topk(out["F"], rank, dt, A, C, k)
    lam0, U0 = bistochastic_evd(ref["F"])
    erel, ang = compare_eigpairs(lam0[:k], U0[:, :k], ev.cpu().numpy(), U.cpu().numpy().T, rel_gap=1e-6,
                                 lam_full=lam0)
    assert erel < 1e-10, erel
    assert ang < 1e-8, ang


def test_paper131k_precision_against_replay(kevd):
    X, eps, cfg = make_config("paper131k")
    rank, ferr, erel, trel = _precision_vs_replay(kevd, X, eps, 1024, cfg["b"], cfg["k"], 1008)
    assert rank > 512, rank
    assert ferr < 1e-3, ferr
    assert erel < 1e-4, erel
    assert trel < 1e-3, trel
