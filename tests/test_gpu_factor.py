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


@pytest.mark.parametrize("N,d,r,b", [(20000, 64, 512, 64), (6001, 64, 300, 128), (3000, 128, 96, 32)])
def test_tensor_core_engine_matches_fp64_pipe(kevd, monkeypatch, N, d, r, b):
    """The FP64 engine with its products on the tensor cores (FP64-accurate digit
    slices, the default) against the FP64-pipe engine (KEVD_ENGINE=fp64) on the same
    input: identical pivots, and F and rho at the FP64 path's bar (1e-10 absolute: two
    FP64 computations with different rounding, whose late columns are amplified by
    1/L_jj; measured 1.7e-11); and against the oracle's replayed factor of those
    pivots at the same bar."""
    from oracle.pchol import pchol_given_pivots
    X, eps, _ = make_config("ks200k" if d == 64 else "vsa2m", N=N)
    Xg = _gpu(X.astype(np.float64))
    oz = kevd.rpchol_factor(Xg, eps, r, mode="arpc", b=b, seed=31)
    monkeypatch.setenv("KEVD_ENGINE", "fp64")
    fp = kevd.rpchol_factor(Xg, eps, r, mode="arpc", b=b, seed=31)
    monkeypatch.delenv("KEVD_ENGINE")
    rk = oz["rank"]
    S = oz["pivots"].cpu().numpy()[:rk]
    assert rk == fp["rank"] and S.tolist() == fp["pivots"].cpu().numpy()[: fp["rank"]].tolist()
    F = oz["F"].cpu().numpy().T[:, :rk]
    assert np.max(np.abs(F - fp["F"].cpu().numpy().T[:, :rk])) < 1e-10
    assert np.max(np.abs(oz["rho"].cpu().numpy() - fp["rho"].cpu().numpy())) < 1e-10
    rp = pchol_given_pivots(X.astype(np.float64), eps, S, blocks=[16] * (rk // 16) + [rk % 16] * (rk % 16 > 0))
    assert np.max(np.abs(F - rp["F"])) < 1e-10


@pytest.mark.parametrize("N,r,k,pad", [(20000, 400, 64, 0), (5001, 129, 40, 1), (30000, 300, 256, 0)])
def test_tensor_core_lift_matches_fp64_pipe(kevd, monkeypatch, N, r, k, pad):
    """The FP64 lift U = D~^-1 F Y on the tensor cores against the FP64-pipe GEMM
    (KEVD_LIFT=fp64) with the same r x r stage: eigenvalues identical, U to 1e-11
    of each column's largest entry (two FP64 products whose rounding differs; Y's
    entries reach ~1e3, so U's cancellation amplifies it), F as a view with
    leading dimension N + pad."""
    X, eps, _ = make_config("ks200k", N=N)
    F = arpc(X, eps, r, 32, 9)["F"]
    rk = F.shape[1]
    k = min(k, rk)
    Fbuf = torch.full((rk, N + pad), float("nan"), dtype=torch.float64)
    Fbuf[:, :N] = torch.from_numpy(np.ascontiguousarray(F.T))
    Fg = Fbuf.cuda()[:, :N]
    dt, qt, A, C = kevd.bistoch_normalize(Fg, rk)
    ev1, U1, _ = kevd.eig_topk(Fg, rk, dt, A, C, k)
    monkeypatch.setenv("KEVD_LIFT", "fp64")
    ev2, U2, _ = kevd.eig_topk(Fg, rk, dt, A, C, k)
    monkeypatch.delenv("KEVD_LIFT")
    assert torch.equal(ev1, ev2)
    U1 = U1.cpu().numpy()
    U2 = U2.cpu().numpy()
    scale = np.max(np.abs(U2), axis=1, keepdims=True)
    assert np.max(np.abs(U1 - U2) / scale) < 1e-11


def test_engine_exp_matches_cuda_exp(kevd):
    """The FP64 engine's table-driven exponential (integer-pipe polynomial) against
    CUDA's exp on t <= 0: within one ulp (relative 2^-52) on a sweep over
    [-708, 0] with the ends and tiny arguments, 1 at t = 0, 0 for t <= -708."""
    g = torch.Generator().manual_seed(5)
    t = torch.cat([-708.0 * torch.rand(400_000, generator=g, dtype=torch.float64),
                   -torch.rand(100_000, generator=g, dtype=torch.float64),
                   -(10.0 ** (-20 * torch.rand(50_000, generator=g, dtype=torch.float64))),
                   torch.tensor([0.0, -0.0, -1e-300, -5e-324, -2 ** -53, -707.999, -1.0, -0.5])]).cuda()
    ours = kevd.kernel_exp(t)
    ref = torch.exp(t)
    rel = ((ours - ref).abs() / ref).max().item()
    assert rel <= 2.0 ** -52, rel
    assert ours[t == 0].eq(1.0).all()
    low = torch.tensor([-708.0, -709.5, -745.2, -1e4, -float("inf")], dtype=torch.float64).cuda()
    assert kevd.kernel_exp(low).eq(0.0).all()
