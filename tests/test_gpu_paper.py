"""The paper-shaped workloads of Section 4 on the GPU (-m gpu).

* paper32k (Section 4.1's set-up: the paper's initial condition, J = 64 delays at one
  grid point, eps = 32 J): the precision form end to end against the FP64 oracle on the
  replayed factor of the GPU's pivots (top-64 eigenvalues within 1e-4 relative).
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
    erel = np.max(np.abs(ev.cpu().numpy() - lam0) / np.abs(lam0))
    F = out["F"].cpu().numpy().astype(np.float64).T[:, :rank]
    return rank, np.max(np.abs(F - rp["F"])), erel


def test_paper32k_precision_against_replay(kevd):
    X, eps, cfg = make_config("paper32k")
    # eps = 32 J leaves a numerical rank near 300; the stopping floor sum(rho) <= 1e-5 N stops
    # the FP32 factor there (past it, FP32-noise pivots can make d~ non-positive: reading 6)
    rank, ferr, erel = _precision_vs_replay(kevd, X, eps, cfg["r"], cfg["b"], cfg["k"], 1006, tol=1e-5)
    assert 100 < rank < cfg["r"], rank
    assert ferr < 1e-3, ferr
    assert erel < 1e-4, erel


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
    rank, ferr, erel = _precision_vs_replay(kevd, X, eps, 1024, cfg["b"], cfg["k"], 1008)
    assert rank > 512, rank
    assert ferr < 1e-3, ferr
    assert erel < 1e-4, erel
