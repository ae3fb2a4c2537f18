"""GPU parity of the FP64 path against the oracle, through the C-ABI (-m gpu).

Inputs are seeded synthetic KS point clouds.  Pivot sequences must match the
oracle exactly (the random draws come from Philox on both sides); a mismatch
is only tolerated at a draw whose oracle-side margin to a CDF edge (or to the
accept threshold) is below 1e-9, which the test reports.
"""
import numpy as np
import pytest
import torch

from datagen import make_config
from oracle.pchol import pchol_given_pivots, greedy_pchol, arpc
from oracle.kernel import kernel_dense
from tests.helpers import first_divergence

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


def test_greedy_ks2k_matches_oracle(kevd):
    X, eps, cfg = make_config("ks2k")
    F0, S0, rho0, _ = greedy_pchol(X, eps, 128)
    out = kevd.rpchol_factor(_gpu(X), eps, 128, mode="greedy")
    assert out["rank"] == len(S0) == 128
    S = out["pivots"].cpu().numpy()
    assert S.tolist() == S0.tolist()
    F = out["F"].cpu().numpy().T
    assert np.max(np.abs(F - F0)) < 1e-12
    assert np.max(np.abs(out["rho"].cpu().numpy() - rho0)) < 1e-12
    assert abs(out["trace_err"] - rho0.sum()) < 1e-10 * 2000
    assert abs(out["trace_err"] - (2000 - np.sum(F * F))) < 1e-9


@pytest.mark.parametrize("N,d,r,b,seed", [(5000, 64, 256, 32, 1002), (1037, 64, 100, 24, 7), (3000, 64, 128, 64, 11)])
def test_arpc_matches_oracle(kevd, N, d, r, b, seed):
    X, eps, _ = make_config("ks200k", N=N)
    ref = arpc(X, eps, r, b, seed)
    out = kevd.rpchol_factor(_gpu(X), eps, r, mode="arpc", b=b, seed=seed, record_proposals=True)
    props = out["proposals"].cpu().numpy()
    diverged = False
    for rnd, lg in enumerate(ref["log"]):
        if rnd >= len(props) or props[rnd].tolist() != lg["proposals"].tolist():
            # a draw within 1e-9 of a CDF or accept edge may resolve either way
            # under another summation order; then check against the replay
            assert _near_edge(ref["log"], rnd), "round %d proposals differ away from a CDF edge" % rnd
            diverged = True
            break
    S = out["pivots"].cpu().numpy()[: out["rank"]]
    if diverged:
        cmp = pchol_given_pivots(X, eps, S, blocks=[16] * (len(S) // 16) + [len(S) % 16] * (len(S) % 16 > 0))
    else:
        assert out["rounds"] == ref["rounds"] == len(ref["log"])
        i = first_divergence(S, ref["pivots"])
        assert i is None, "pivot %d differs" % i
        cmp = ref
    F = out["F"].cpu().numpy().T[:, : out["rank"]]
    assert np.max(np.abs(F - cmp["F"])) < 1e-10
    rho = out["rho"].cpu().numpy()
    assert np.max(np.abs(rho - cmp["rho"])) < 1e-10
    assert abs(out["trace_err"] - cmp["rho"].sum()) <= 1e-10 * N
    # columns past the rank are zero
    assert np.all(out["F"].cpu().numpy()[out["rank"]:] == 0)


def test_arpc_until_rank(kevd):
    X, eps, _ = make_config("ks200k", N=2000)
    ref = arpc(X, eps, 96, 32, 5, until_rank=True)
    out = kevd.rpchol_factor(_gpu(X), eps, 96, mode="arpc", b=32, seed=5, until_rank=True)
    assert out["rank"] == 96 == ref["F"].shape[1]
    assert out["pivots"].cpu().numpy().tolist() == ref["pivots"].tolist()
    assert np.max(np.abs(out["F"].cpu().numpy().T - ref["F"])) < 1e-10


def test_deterministic(kevd):
    X, eps, _ = make_config("ks200k", N=4000)
    a = kevd.rpchol_factor(_gpu(X), eps, 128, mode="arpc", b=64, seed=3)
    b = kevd.rpchol_factor(_gpu(X), eps, 128, mode="arpc", b=64, seed=3)
    assert torch.equal(a["F"], b["F"]) and torch.equal(a["rho"], b["rho"])


def test_full_rank_greedy_reproduces_K(kevd):
    rng = np.random.Generator(np.random.PCG64(0))
    X = rng.standard_normal((50, 3))
    out = kevd.rpchol_factor(_gpu(X), 0.3, 50, mode="greedy")
    F = out["F"].cpu().numpy().T
    assert out["rank"] == 50
    assert np.max(np.abs(F @ F.T - kernel_dense(X, 0.3))) < 1e-12


def test_edge_cases(kevd):
    # one point
    out = kevd.rpchol_factor(_gpu(np.zeros((1, 4))), 1.0, 1, mode="greedy")
    assert out["rank"] == 1 and abs(out["F"].item() - 1.0) < 1e-15 and out["trace_err"] == 0.0
    # identical points: one pivot explains everything, rho -> 0, early stop
    X = np.ones((300, 5))
    out = kevd.rpchol_factor(_gpu(X), 1.0, 64, mode="arpc", b=16, seed=1)
    assert out["rank"] == 1 and out["trace_err"] == 0.0
    out = kevd.rpchol_factor(_gpu(X), 1.0, 8, mode="greedy")
    assert out["rank"] == 1
    # d = 1, b = 128 (maximum block)
    X = np.linspace(-3, 3, 700)[:, None]
    ref = arpc(X, 0.5, 256, 128, 9)
    out = kevd.rpchol_factor(_gpu(X), 0.5, 256, mode="arpc", b=128, seed=9)
    assert out["pivots"].cpu().numpy()[: out["rank"]].tolist() == ref["pivots"].tolist()
    assert np.max(np.abs(out["F"].cpu().numpy().T[:, : out["rank"]] - ref["F"])) < 1e-10


def test_bad_inputs(kevd):
    X = np.zeros((100, 3))
    X[17, 1] = np.nan
    with pytest.raises(kevd.KevdError) as e:
        kevd.rpchol_factor(_gpu(X), 1.0, 8, mode="greedy")
    assert e.value.status == 1
    with pytest.raises(kevd.KevdError):
        kevd.rpchol_factor(_gpu(np.zeros((10, 2))), -1.0, 4, mode="greedy")


def test_tol_floor_stops_early(kevd):
    X, eps, _ = make_config("ks200k", N=3000)
    full = kevd.rpchol_factor(_gpu(X), eps, 256, mode="arpc", b=32, seed=2)
    tol = 0.05
    out = kevd.rpchol_factor(_gpu(X), eps, 256, mode="arpc", b=32, seed=2, tol=tol)
    # identical rounds until the floor, then no further pivots
    assert out["rank"] < full["rank"]
    assert torch.equal(out["pivots"][: out["rank"]], full["pivots"][: out["rank"]])
    assert out["trace_err"] <= tol * 3000 * 1.0000001
