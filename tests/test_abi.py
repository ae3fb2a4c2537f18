"""The C-ABI library builds, loads and exports every symbol of include/kevd.h;
argument errors are reported before any device work (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2510_26574_gb300 as kevd
from paper_2510_26574_gb300 import kevd as K
from paper_2510_26574_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return kevd.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "kevd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**([A-Za-z_]\w*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert set(names) == set(kevd.EXPORTS), names
    for n in names:
        assert hasattr(L, n)


def test_status_strings(L):
    for code in (0, 1, 2, 3, 4, 5, 7):
        assert kevd.status_string(code) and kevd.status_string(code) != "unknown status"
    assert kevd.status_string(99) == "unknown status"


def test_factor_workspace_size(L):
    o = K.make_opts("arpc", 64, 1)
    n1 = K.workspace_bytes(K.KEVD_WS_FACTOR, 200000, 64, 1024, 1, o)
    n2 = K.workspace_bytes(K.KEVD_WS_FACTOR, 400000, 64, 1024, 1, o)
    assert n1 > 0 and n2 > n1
    assert K.workspace_bytes(K.KEVD_WS_FACTOR, 0, 64, 10, 1, o) == 0
    assert K.workspace_bytes(K.KEVD_WS_FACTOR, 100, 64, 10, 1, K.make_opts("arpc", 129, 1)) == 0
    assert K.workspace_bytes(K.KEVD_WS_NORMALIZE, 100, 1, 200) == 0      # rank > N


def test_argument_errors_before_device_work(L):
    dummy = ctypes.c_void_p(16)            # never dereferenced: validation fails first
    info = K.kevd_factor_info()
    o = K.make_opts("arpc", 64, 1)
    ws = ctypes.c_void_p(256)

    def call(X=dummy, N=1000, d=8, eps=1.0, r=64, opts=o, ldf=1000, wsb=0, xdt=K.KEVD_F64):
        return L.rpchol_factor(X, xdt, N, d, eps, r, ctypes.byref(opts), dummy, K.KEVD_F64, ldf, dummy, dummy,
                               None, ctypes.byref(info), ws, wsb, None)

    assert call(X=None) == K.KEVD_EINVAL
    assert call(eps=0.0) == K.KEVD_EINVAL
    assert call(eps=float("nan")) == K.KEVD_EINVAL
    assert call(r=1001) == K.KEVD_EINVAL
    assert call(ldf=999) == K.KEVD_EINVAL
    assert call(opts=K.make_opts("arpc", 200, 1)) == K.KEVD_EINVAL
    assert call(opts=K.make_opts("arpc", 128, 1), r=64) == K.KEVD_EINVAL    # t = r/b = 0 rounds
    assert call(opts=K.make_opts("arpc", 64, 1, tol=1.5)) == K.KEVD_EINVAL
    assert call(wsb=16) == K.KEVD_EWORKSPACE
    assert L.bistoch_normalize(dummy, K.KEVD_F64, 10, 20, 10, dummy, dummy, dummy, dummy, ws, 0, None) == K.KEVD_EINVAL
    assert L.bistoch_normalize(dummy, K.KEVD_F64, 100, 20, 100, dummy, dummy, dummy, dummy, ws, 16, None) == K.KEVD_EWORKSPACE
    kept = ctypes.c_int32(0)
    assert L.eig_topk(dummy, K.KEVD_F64, 100, 20, 100, dummy, dummy, dummy, 21, 1e-13, dummy, dummy,
                      ctypes.byref(kept), ws, 0, None) == K.KEVD_EINVAL
    assert L.eig_topk(dummy, K.KEVD_F64, 100, 20, 100, dummy, dummy, dummy, 4, 1.5, dummy, dummy,
                      ctypes.byref(kept), ws, 0, None) == K.KEVD_EINVAL


def test_lowmem_workspace_size(L, monkeypatch):
    """The low-memory factor's workspace is O(N + P r + r d + r b), far below the N x r factor."""
    o = K.make_opts("arpc", 64, 1)
    N, d, r = 2_000_000, 64, 2048
    n_lm = K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, N, d, r, 1, o)
    monkeypatch.setenv("KEVD_ENGINE", "fp64")                 # the stored-F round state without product arrays
    n_fp = K.workspace_bytes(K.KEVD_WS_FACTOR, N, d, r, 1, o)
    monkeypatch.delenv("KEVD_ENGINE")
    assert n_lm > n_fp                                        # the FP64 round state plus one panel
    assert n_lm - n_fp < (1 << 27) + 8 * (r * d + r + r * 64) + 8 * 256   # panel <= 128 MiB
    assert n_lm < N * r * 8 // 100                            # < 1% of the FP64 factor itself
    n_norm = K.workspace_bytes(K.KEVD_WS_LOWMEM_NORMALIZE, N, d, r)
    assert 0 < n_norm < N * r * 8 // 100
    assert K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, 100, 8, 200, 1, o) == 0   # r > N
    assert K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, 100, 8, 10, 1, None) == 0
    assert K.workspace_bytes(K.KEVD_WS_LOWMEM_NORMALIZE, 100, 0, 10) == 0


def test_lowmem_argument_errors_before_device_work(L):
    dummy = ctypes.c_void_p(16)
    info = K.kevd_factor_info()
    o = K.make_opts("arpc", 64, 1)
    ws = ctypes.c_void_p(256)

    def call(X=dummy, N=1000, d=8, eps=1.0, r=64, opts=o, ldw=64, wsb=0):
        return L.rpchol_factor_lowmem(X, N, d, eps, r, ctypes.byref(opts), dummy, ldw, dummy, dummy, None,
                                      ctypes.byref(info), ws, wsb, None)

    assert call(X=None) == K.KEVD_EINVAL
    assert call(eps=-1.0) == K.KEVD_EINVAL
    assert call(r=1001) == K.KEVD_EINVAL
    assert call(ldw=63) == K.KEVD_EINVAL
    assert call(opts=K.make_opts("arpc", 64, 1, precision=K.KEVD_PREC_BF16X3)) == K.KEVD_EINVAL   # FP64 only
    assert call(opts=K.make_opts("arpc", 128, 1)) == K.KEVD_EINVAL                               # 0 rounds
    assert call(wsb=16) == K.KEVD_EWORKSPACE
    assert L.bistoch_normalize_lowmem(dummy, 100, 8, 1.0, dummy, dummy, 10, 20, dummy, dummy, dummy, dummy, ws, 0,
                                      None) == K.KEVD_EINVAL                                    # ldw < rank
    assert L.bistoch_normalize_lowmem(dummy, 100, 8, 1.0, dummy, dummy, 20, 20, dummy, dummy, dummy, dummy, ws, 16,
                                      None) == K.KEVD_EWORKSPACE
    kept = ctypes.c_int32(0)
    assert L.eig_topk_lowmem(dummy, 100, 8, 1.0, dummy, dummy, 20, 20, dummy, dummy, dummy, 21, 1e-13, dummy, dummy,
                             ctypes.byref(kept), ws, 0, None) == K.KEVD_EINVAL                 # k > rank
    assert L.eig_topk_lowmem(dummy, 100, 8, 0.0, dummy, dummy, 20, 20, dummy, dummy, dummy, 4, 1e-13, dummy, dummy,
                             ctypes.byref(kept), ws, 0, None) == K.KEVD_EINVAL                 # eps = 0


def test_lowmem_panel_rule(L, monkeypatch):
    """Panel rows P = min(N rounded up to 64, floor(2^24 / r) rounded down to 64, >= 64);
    KEVD_LOWMEM_PANEL lowers the 2^24 / r rule and cannot raise it.  Only the P x r panel depends on P."""
    o = K.make_opts("arpc", 16, 1)
    N, d, r = 10000, 8, 100
    monkeypatch.delenv("KEVD_LOWMEM_PANEL", raising=False)
    base = K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, N, d, r, 1, o)
    monkeypatch.setenv("KEVD_LOWMEM_PANEL", "256")
    small = K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, N, d, r, 1, o)
    assert base - small == (10048 - 256) * r * 8          # default P = N rounded up to 64
    monkeypatch.setenv("KEVD_LOWMEM_PANEL", "300")          # rounded down to 256
    assert K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, N, d, r, 1, o) == small
    monkeypatch.setenv("KEVD_LOWMEM_PANEL", "10")           # at least 64 rows
    tiny = K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, N, d, r, 1, o)
    assert small - tiny == (256 - 64) * r * 8
    monkeypatch.delenv("KEVD_LOWMEM_PANEL")
    r2 = 4096                                               # 2^24 / 4096 = 4096 rows
    n2 = 100000
    big = K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, n2, d, r2, 1, o)
    monkeypatch.setenv("KEVD_LOWMEM_PANEL", "4096")
    assert K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, n2, d, r2, 1, o) == big
    monkeypatch.setenv("KEVD_LOWMEM_PANEL", "1000000")     # above the rule: capped at 4096 rows
    assert K.workspace_bytes(K.KEVD_WS_LOWMEM_FACTOR, n2, d, r2, 1, o) == big


def test_noalloc_path_names_no_allocating_call():
    """rpchol_factor_noalloc runs rpchol_factor (factor.cu, both engines) on a
    static array: none of these sources may name a device allocation or a
    library handle constructor (which allocates)."""
    import re
    csrc = os.path.join(ROOT, "paper_2510_26574_gb300", "csrc")
    banned = re.compile(r"cudaMalloc|cudaFree|cudaMallocAsync|cublasCreate|cusolverDnCreate|cudaMallocManaged")
    for f in ("noalloc.cu", "factor.cu", "factor.cuh", "engine_tc.cu", "tc_ptx.cuh", "common.cuh"):
        src = open(os.path.join(csrc, f)).read()
        assert not banned.search(src), f


def test_opts_init_defaults(L):
    """kevd_opts_init gives every field its documented default; the precision
    form's stopping floor comes from the library, not from the binding."""
    o = K.kevd_opts()
    ctypes.memset(ctypes.byref(o), 0xFF, ctypes.sizeof(o))
    L.kevd_opts_init(ctypes.byref(o), K.KEVD_PREC_BF16X3)
    assert (o.mode, o.precision, o.block_b, o.until_rank, o.max_rounds, o.reserved, o.seed) == (
        K.KEVD_ARPC, K.KEVD_PREC_BF16X3, 64, 0, 0, 0, 0)
    assert o.tol == 1e-6
    L.kevd_opts_init(ctypes.byref(o), K.KEVD_PREC_FP64)
    assert o.precision == K.KEVD_PREC_FP64 and o.tol == 0.0
    assert K.make_opts("arpc", 32, 5, precision="bf16x3").tol == 1e-6
    assert K.make_opts("arpc", 32, 5, precision="bf16x3", tol=0.0).tol == 0.0


def test_fp64_factor_workspace_holds_tensor_core_products(L, monkeypatch):
    """The FP64 factor runs its engine on the tensor cores by default (ARPC, b >= 32):
    the workspace adds two N x b FP64 product arrays, seven BF16 digit planes of X
    (N x round16(d)), of F (N x round16(r + 15 rounds): each round's columns padded to
    16), of R and of the pivot panels and L^-1, the row exponents and the FP64 inverse
    over the FP64-pipe engine's (KEVD_ENGINE=fp64)."""
    o = K.make_opts("arpc", 64, 1)
    N, d, r, b = 100_001, 64, 1024, 64
    full = K.workspace_bytes(K.KEVD_WS_FACTOR, N, d, r, 1, o)
    monkeypatch.setenv("KEVD_ENGINE", "fp64")
    base = K.workspace_bytes(K.KEVD_WS_FACTOR, N, d, r, 1, o)
    rounds = r // b
    ldD, ldX, ldR, ldLi = N + 1, 64, 64, 64
    ldF = (r + 15 * rounds + 15) // 16 * 16
    planes = 14 * (N * ldX + N * ldF + N * ldR + b * ldX + b * ldF + b * ldR)
    extra = 16 * ldD * b + planes + 4 * (2 * N + 2 * b) + 8 * b * ldLi + 16
    assert 0 < full - base - extra < 15 * 256                 # each carve rounds up to 256 bytes
    p = K.make_opts("arpc", 64, 1, precision=K.KEVD_PREC_BF16X3)
    prec = K.workspace_bytes(K.KEVD_WS_FACTOR, N, d, r, 1, p)
    g = K.make_opts("greedy", 1, 1)
    greedy = K.workspace_bytes(K.KEVD_WS_FACTOR, N, d, r, 1, g)
    monkeypatch.delenv("KEVD_ENGINE")
    assert K.workspace_bytes(K.KEVD_WS_FACTOR, N, d, r, 1, p) == prec     # the precision form has none
    assert K.workspace_bytes(K.KEVD_WS_FACTOR, N, d, r, 1, g) == greedy   # nor greedy (b = 1)