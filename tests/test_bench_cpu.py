"""The bench's work accounting, checked on the CPU against brute-force sums.

The roofline divides algorithmic work by traced stage times.  The work comes
from the factor's counters (rank, sum_k = sum over engine rounds of the rank
before the round, sum_m_sq = sum of m^2), so the closed forms are checked here
against a direct sum over a simulated sequence of rounds.
"""
import numpy as np
import pytest

import bench


def _rounds(seed, n_rounds, b):
    rng = np.random.Generator(np.random.PCG64(seed))
    m = rng.integers(0, b + 1, n_rounds)
    k = np.concatenate([[0], np.cumsum(m)[:-1]])
    eng = m > 0
    out = dict(rank=int(m.sum()), sum_m_sq=int((m * m).sum()), sum_k=int(k[eng].sum()),
               engine_rounds=int(eng.sum()), rounds=n_rounds)
    return m, k, out


def _stages(eng_ms=100.0, gram_ms=50.0, steps=1):
    s = {n: (0.0, 0) for n in bench.STAGE_NAMES} if hasattr(bench, "STAGE_NAMES") else {}
    s.update({"engine": (eng_ms * steps, steps), "gram": (gram_ms * steps, steps)})
    return s


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lowmem_factor_work_closed_form(seed):
    N, d, b = 1000, 64, 64
    m, k, out = _rounds(seed, 16, b)
    brute = sum(N * (2.0 * d * (ki + mi) + 2.0 * ki * mi + mi * mi) for ki, mi in zip(k, m) if mi > 0)
    cfg = dict(N=N, d=d)
    rf = bench.roofline("lowmem", _stages(eng_ms=1000.0, gram_ms=1e-3), out, cfg, 1)
    name = [n for n in rf["stages"] if n.startswith("factor")][0]
    assert rf["stages"][name]["gflop"] * 1e9 == pytest.approx(brute, rel=1e-12)
    assert rf["kernel"] == name                       # the slower stage is the one reported
    assert rf["achieved"] == pytest.approx(brute / 1.0 / 1e9, rel=1e-12)


@pytest.mark.parametrize("seed", [3, 4])
def test_fp64_engine_work_closed_form(seed):
    N, d, b = 500, 32, 32
    m, k, out = _rounds(seed, 12, b)
    brute = sum(N * (2.0 * d * mi + 2.0 * ki * mi + mi * mi) for ki, mi in zip(k, m))
    rank = out["rank"]
    closed = N * (2.0 * d * rank + float(rank) ** 2)    # 2 sum k m = rank^2 - sum m^2
    assert closed == pytest.approx(brute, rel=1e-12)
    rf = bench.roofline("fp64", _stages(eng_ms=1000.0, gram_ms=1e-3), out, dict(N=N, d=d), 1)
    assert rf["kernel"] == "k_engine"
    assert rf["achieved"] == pytest.approx(brute / 1e9, rel=1e-12)


def test_lowmem_launch_count_grows_with_panels():
    out = dict(rank=801, rounds=16, engine_rounds=16, sum_k=5358, sum_m_sq=42005)
    small = bench.lowmem_launches(20000, out, 1)
    large = bench.lowmem_launches(200000, out, 1)
    assert 0 < small < large
    assert bench.lowmem_launches(200000, out, 3) == 3 * large


@pytest.mark.filterwarnings("ignore:CUDA is not available")
def test_counted_launches_reports_why_instead_of_raising(monkeypatch):
    """The launch count is informational: without a GPU (no kernel, or synchronize fails)
    and under another CUDA profiler it returns no count and a reason, never an exception."""
    monkeypatch.delenv("CUDA_INJECTION64_PATH", raising=False)
    n, why = bench.counted_launches(lambda _x: None, None)
    assert n is None and why
    monkeypatch.setenv("CUDA_INJECTION64_PATH", "/nonexistent/injection.so")
    calls = []
    n, why = bench.counted_launches(lambda _x: calls.append(1), None)
    assert n is None and "profiler" in why and not calls   # the step is not even run
