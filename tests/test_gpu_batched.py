"""Batched form (-m gpu): every problem of the lockstep batched launch (CUDA
graph replay or direct launches) must equal its single-problem rpchol_factor
run with the FP64-pipe engine (KEVD_ENGINE=fp64) bit for bit (the same kernels
compute every output in the same order)."""
import numpy as np
import pytest
import torch

from datagen import make_config, batched_problems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kevd():
    from paper_2510_26574_gb300.build import build
    build()
    import paper_2510_26574_gb300 as m
    return m


def _problems():
    shapes = [(3001, 64, 128, 32, "ks200k"), (1037, 96, 100, 24, "vsa524k"), (5000, 64, 256, 64, "ks200k"),
              (700, 128, 64, 64, "vsa2m"), (2222, 64, 96, 16, "ks200k")]
    probs = []
    for q, (N, d, r, b, name) in enumerate(shapes):
        X, eps, _ = make_config(name, N=N)
        probs.append(dict(X=torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).cuda(), eps=eps * (0.5 + q / 4),
                          r=r, b=b, seed=100 + q))
    return probs


@pytest.mark.parametrize("use_graph", [True, False])
def test_batched_equals_single(kevd, monkeypatch, use_graph):
    monkeypatch.setenv("KEVD_ENGINE", "fp64")
    probs = _problems()
    batch = kevd.Batch(probs, use_graph=use_graph)
    for rep in range(2):                                  # replay twice
        outs = batch.run()
        for p, o in zip(probs, outs):
            ref = kevd.rpchol_factor(p["X"], p["eps"], p["r"], mode="arpc", b=p["b"], seed=p["seed"])
            assert o["rank"] == ref["rank"] and o["rounds"] == ref["rounds"]
            assert torch.equal(o["pivots"][: o["rank"]], ref["pivots"][: ref["rank"]])
            assert torch.equal(o["F"], ref["F"])
            assert torch.equal(o["rho"], ref["rho"])
            assert o["trace_err"] == ref["trace_err"]
    batch.close()


def test_batched_config_shapes(kevd, monkeypatch):
    """Uneven Gaussian-mixture problems of the batched workload (first 6), autotuned b."""
    monkeypatch.setenv("KEVD_ENGINE", "fp64")
    from paper_2510_26574_gb300.autotune import tune
    raw = batched_problems(6, n_range=(5000, 20000), r_range=(128, 256))
    probs = [dict(X=torch.from_numpy(p["X"]).cuda(), eps=p["eps"], r=p["r"], b=p["b"], seed=p["seed"]) for p in raw]
    bs = tune(probs, use_cache=False)
    assert all(b in (16, 32, 64, 128) and b <= p["r"] for b, p in zip(bs, probs))
    for p, b in zip(probs, bs):
        p["b"] = b
    outs = kevd.Batch(probs).run()
    for p, o in zip(probs, outs):
        ref = kevd.rpchol_factor(p["X"], p["eps"], p["r"], mode="arpc", b=p["b"], seed=p["seed"])
        assert torch.equal(o["F"], ref["F"])
        N = p["X"].shape[0]
        F = o["F"].cpu().numpy()[: o["rank"]]
        assert abs(o["trace_err"] - (N - np.sum(F * F))) < 1e-8 * N


def test_batched_members_against_oracle(kevd):
    """Three members of the batched workload (uneven N, d, eps, r) end to end: the batch's
    factor of each against the FP64 oracle's replay of its pivots (Algorithm 2), and the
    top-16 eigenvalues of its normalisation and eigensolve against Algorithm 1 on the
    oracle's factor, at the FP64 path's bars."""
    from oracle.pchol import pchol_given_pivots
    from oracle.alg1 import bistochastic_evd
    raw = batched_problems(3, seed=11, n_range=(6000, 12000), r_range=(128, 256))
    probs = [dict(X=torch.from_numpy(p["X"]).cuda(), eps=p["eps"], r=p["r"], b=p["b"], seed=p["seed"]) for p in raw]
    batch = kevd.Batch(probs)
    outs = batch.run()
    for p, q, o in zip(raw, probs, outs):
        rank = o["rank"]
        S = o["pivots"].cpu().numpy()[:rank]
        rp = pchol_given_pivots(p["X"], p["eps"], S, blocks=[16] * (rank // 16) + [rank % 16] * (rank % 16 > 0))
        F = o["F"].cpu().numpy().T[:, :rank]
        assert np.max(np.abs(F - rp["F"])) < 1e-10
        dt, qt, A, C = kevd.bistoch_normalize(o["F"], rank)
        ev, U, kept = kevd.eig_topk(o["F"], rank, dt, A, C, 16)
        lam0, _ = bistochastic_evd(rp["F"], 16)
        erel = np.max(np.abs(ev.cpu().numpy() - lam0) / np.abs(lam0))
        assert erel < 1e-10, (p["N"], p["d"], rank, erel)
    batch.close()
