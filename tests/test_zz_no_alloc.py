"""rpchol_factor_noalloc: the factorisation for callers that cannot allocate
device memory (for example a plugin whose host application owns every device
allocation, or a process that may not allocate after start-up).  Its workspace
is a fixed static device array inside the library, so this test calls it
through the C-ABI and checks that two calls in a row reproduce the output of
rpchol_factor (which takes a caller-allocated workspace) within the FP64
tolerance of the other parity tests, and that sizes beyond the array are
rejected.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    from paper_2510_26574_gb300.build import build
    build()
    from paper_2510_26574_gb300 import kevd
    kevd.lib()
    return kevd


def _call_noalloc(K, Xg, eps, r, opts, F, piv, rho):
    info = K.kevd_factor_info()
    N, d = Xg.shape
    code = K.KEVD_F32 if Xg.dtype == torch.float32 else K.KEVD_F64
    st = K.lib().rpchol_factor_noalloc(K._ptr(Xg), code, N, d, float(eps), r, ctypes.byref(opts), K._ptr(F),
                                       code, N, K._ptr(piv), K._ptr(rho), None, ctypes.byref(info),
                                       K._stream(Xg.device))
    return st, info


def test_noalloc_matches_workspace_entry_point(K, monkeypatch):
    # the no-workspace entry point keeps the FP64 engine's products on the FP64
    # pipe, which rpchol_factor also runs under KEVD_ENGINE=fp64
    monkeypatch.setenv("KEVD_ENGINE", "fp64")
    from datagen import make_config
    X, eps, _ = make_config("ks200k", N=6000)
    Xg = torch.from_numpy(X).cuda()
    r, b, seed = 192, 32, 17
    ref = K.rpchol_factor(Xg, eps, r, mode="arpc", b=b, seed=seed)
    opts = K.make_opts("arpc", b, seed)
    for _ in range(2):                                  # two calls in a row share the static scratch
        F = torch.full((r, 6000), np.nan, dtype=torch.float64, device="cuda")
        piv = torch.full((r,), -1, dtype=torch.int64, device="cuda")
        rho = torch.full((6000,), np.nan, dtype=torch.float64, device="cuda")
        st, info = _call_noalloc(K, Xg, eps, r, opts, F, piv, rho)
        torch.cuda.synchronize()
        assert st == K.KEVD_OK, K.status_string(st)
        assert info.rank == ref["rank"] and info.rounds == ref["rounds"]
        assert torch.equal(piv[: info.rank], ref["pivots"][: ref["rank"]])
        assert torch.max(torch.abs(F - ref["F"])).item() < 1e-12
        assert torch.max(torch.abs(rho - ref["rho"])).item() < 1e-12
        assert abs(info.trace_err - ref["trace_err"]) < 1e-12 * 6000


def test_noalloc_greedy_twice(K, monkeypatch):
    monkeypatch.setenv("KEVD_ENGINE", "fp64")
    from datagen import make_config
    X, eps, _ = make_config("ks2k", N=1500)
    Xg = torch.from_numpy(X).cuda()
    ref = K.rpchol_factor(Xg, eps, 64, mode="greedy")
    opts = K.make_opts("greedy")
    for _ in range(2):
        F = torch.empty((64, 1500), dtype=torch.float64, device="cuda")
        piv = torch.empty(64, dtype=torch.int64, device="cuda")
        rho = torch.empty(1500, dtype=torch.float64, device="cuda")
        st, info = _call_noalloc(K, Xg, eps, 64, opts, F, piv, rho)
        torch.cuda.synchronize()
        assert st == K.KEVD_OK
        assert torch.equal(piv, ref["pivots"])
        assert torch.max(torch.abs(F - ref["F"])).item() < 1e-12


def test_noalloc_precision_form_twice(K):
    """The precision form (FP32 X and F, tensor-core split products) carves a
    different layout into the same static array (pivot panels, FP32 L, an error
    flag); two calls in a row must still reproduce rpchol_factor.  The engine is
    deterministic, so the pivots are identical and F agrees to FP32 rounding."""
    from datagen import make_config
    X, eps, _ = make_config("vsa2m", N=4000)
    X32 = np.ascontiguousarray(X, dtype=np.float32)
    Xg = torch.from_numpy(X32).cuda()
    r, b, seed = 128, 64, 23
    ref = K.rpchol_factor(Xg, eps, r, mode="arpc", b=b, seed=seed)
    opts = K.make_opts("arpc", b, seed, precision=K.KEVD_PREC_BF16X3)
    for _ in range(2):
        F = torch.full((r, 4000), np.nan, dtype=torch.float32, device="cuda")
        piv = torch.full((r,), -1, dtype=torch.int64, device="cuda")
        rho = torch.full((4000,), np.nan, dtype=torch.float64, device="cuda")
        st, info = _call_noalloc(K, Xg, eps, r, opts, F, piv, rho)
        torch.cuda.synchronize()
        assert st == K.KEVD_OK, K.status_string(st)
        assert info.rank == ref["rank"] and info.rounds == ref["rounds"]
        assert torch.equal(piv[: info.rank], ref["pivots"][: ref["rank"]])
        assert torch.max(torch.abs(F - ref["F"])).item() < 1e-6
        assert torch.max(torch.abs(rho - ref["rho"])).item() < 1e-9


def test_noalloc_rejects_sizes_beyond_scratch(K):
    opts = K.make_opts("arpc", 64, 1)
    assert K.workspace_bytes(K.KEVD_WS_FACTOR, 4_000_000, 8, 64, 1, opts) > K.KEVD_NOALLOC_SCRATCH_BYTES
    dummy = ctypes.c_void_p(256)                         # never dereferenced: rejected before any work
    info = K.kevd_factor_info()
    st = K.lib().rpchol_factor_noalloc(dummy, K.KEVD_F64, 4_000_000, 8, 1.0, 64, ctypes.byref(opts), dummy,
                                       K.KEVD_F64, 4_000_000, dummy, dummy, None, ctypes.byref(info), None)
    assert st == K.KEVD_ESCRATCH
    assert "static scratch" in K.status_string(st)
