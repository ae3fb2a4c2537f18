"""Python binding of libkevd (ctypes): argument marshalling only.

The functions keep the C-ABI names.  PyTorch supplies device memory (outputs
and workspace are torch tensors on the input's device) and the current CUDA
stream; every step of the computation runs in libkevd's kernels.  There is no
fallback: if libkevd.so is missing or a call fails, an exception is raised.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkevd.so")

KEVD_OK, KEVD_EINVAL, KEVD_ED_NONPOS, KEVD_EQ_NONPOS, KEVD_ECUDA, KEVD_EWORKSPACE, KEVD_EEIG = 0, 1, 2, 3, 4, 5, 7
KEVD_ESCRATCH = 8
KEVD_NOALLOC_SCRATCH_BYTES = 16 << 20
KEVD_F64, KEVD_F32 = 0, 1
KEVD_GREEDY, KEVD_ARPC = 0, 1
KEVD_PREC_FP64, KEVD_PREC_BF16X3 = 0, 1
KEVD_ETIMEOUT = 6
PRECISIONS = {"fp64": KEVD_PREC_FP64, "bf16x3": KEVD_PREC_BF16X3}
KEVD_WS_FACTOR, KEVD_WS_NORMALIZE, KEVD_WS_EIG, KEVD_WS_FIX = 0, 1, 2, 3
KEVD_WS_LOWMEM_FACTOR, KEVD_WS_LOWMEM_NORMALIZE, KEVD_WS_LOWMEM_EIG = 4, 5, 6

# every symbol of include/kevd.h
EXPORTS = ("rpchol_factor", "bistoch_normalize", "eig_topk", "kevd_workspace_bytes", "kevd_status_string",
           "kevd_trace_enable", "kevd_trace_reset", "kevd_trace_read", "rpchol_factor_noalloc",
           "kevd_batch_workspace_bytes", "kevd_batch_create", "kevd_batch_run", "kevd_batch_destroy",
           "symmetric_normalize", "symmetric_eig_topk", "constant_eigvec_fix", "rpchol_factor_lowmem",
           "bistoch_normalize_lowmem", "eig_topk_lowmem", "kevd_opts_init", "kevd_kernel_exp")
STAGES = ("propose", "gather", "blockH", "reject", "engine", "degree", "gram", "solver", "lift", "other", "products")


class kevd_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("block_b", ctypes.c_int32),
                ("until_rank", ctypes.c_int32), ("max_rounds", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("tol", ctypes.c_double)]


class kevd_factor_info(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("rounds", ctypes.c_int32), ("trace_err", ctypes.c_double),
                ("sum_m_sq", ctypes.c_int64), ("sum_k", ctypes.c_int64), ("engine_rounds", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class kevd_problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("d", ctypes.c_int32), ("r", ctypes.c_int32),
                ("b", ctypes.c_int32), ("reserved", ctypes.c_int32), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("F", ctypes.c_void_p), ("ldf", ctypes.c_int64),
                ("pivots", ctypes.c_void_p), ("rho", ctypes.c_void_p)]


class KevdError(RuntimeError):
    def __init__(self, call, status):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (call, status_string(status), status))


_lib = None


def lib():
    """The loaded libkevd.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libkevd.so is not built (run paper_2510_26574_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.rpchol_factor.argtypes = [vp, ctypes.c_int, i64, i32, dbl, i32, ctypes.POINTER(kevd_opts), vp,
                                    ctypes.c_int, i64, vp, vp, vp, ctypes.POINTER(kevd_factor_info), vp,
                                    ctypes.c_size_t, vp]
        L.rpchol_factor.restype = ctypes.c_int
        L.bistoch_normalize.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.bistoch_normalize.restype = ctypes.c_int
        L.eig_topk.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, vp, vp, i32, dbl, vp, vp,
                               ctypes.POINTER(ctypes.c_int32), vp, ctypes.c_size_t, vp]
        L.eig_topk.restype = ctypes.c_int
        L.rpchol_factor_noalloc.argtypes = [vp, ctypes.c_int, i64, i32, dbl, i32, ctypes.POINTER(kevd_opts), vp,
                                            ctypes.c_int, i64, vp, vp, vp, ctypes.POINTER(kevd_factor_info), vp]
        L.rpchol_factor_noalloc.restype = ctypes.c_int
        L.kevd_workspace_bytes.argtypes = [ctypes.c_int, i64, i32, i32, i32, ctypes.POINTER(kevd_opts)]
        L.kevd_workspace_bytes.restype = ctypes.c_size_t
        L.kevd_status_string.argtypes = [ctypes.c_int]
        L.kevd_status_string.restype = ctypes.c_char_p
        L.kevd_batch_workspace_bytes.argtypes = [ctypes.POINTER(kevd_problem), ctypes.c_int]
        L.kevd_batch_workspace_bytes.restype = ctypes.c_size_t
        L.kevd_batch_create.argtypes = [ctypes.POINTER(kevd_problem), ctypes.c_int, ctypes.c_int, vp,
                                        ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_void_p)]
        L.kevd_batch_create.restype = ctypes.c_int
        L.kevd_batch_run.argtypes = [vp, vp, ctypes.POINTER(kevd_factor_info)]
        L.kevd_batch_run.restype = ctypes.c_int
        L.kevd_batch_destroy.argtypes = [vp]
        L.kevd_batch_destroy.restype = None
        L.symmetric_normalize.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, vp, vp, ctypes.c_size_t, vp]
        L.symmetric_normalize.restype = ctypes.c_int
        L.symmetric_eig_topk.argtypes = [vp, ctypes.c_int, i64, i32, i64, vp, vp, i32, vp, vp, vp, ctypes.c_size_t, vp]
        L.symmetric_eig_topk.restype = ctypes.c_int
        L.constant_eigvec_fix.argtypes = [vp, i64, i32, vp, ctypes.c_size_t, vp]
        L.constant_eigvec_fix.restype = ctypes.c_int
        L.rpchol_factor_lowmem.argtypes = [vp, i64, i32, dbl, i32, ctypes.POINTER(kevd_opts), vp, i64, vp, vp, vp,
                                           ctypes.POINTER(kevd_factor_info), vp, ctypes.c_size_t, vp]
        L.rpchol_factor_lowmem.restype = ctypes.c_int
        L.bistoch_normalize_lowmem.argtypes = [vp, i64, i32, dbl, vp, vp, i64, i32, vp, vp, vp, vp, vp,
                                               ctypes.c_size_t, vp]
        L.bistoch_normalize_lowmem.restype = ctypes.c_int
        L.eig_topk_lowmem.argtypes = [vp, i64, i32, dbl, vp, vp, i64, i32, vp, vp, vp, i32, dbl, vp, vp,
                                      ctypes.POINTER(ctypes.c_int32), vp, ctypes.c_size_t, vp]
        L.eig_topk_lowmem.restype = ctypes.c_int
        L.kevd_opts_init.argtypes = [ctypes.POINTER(kevd_opts), ctypes.c_int32]
        L.kevd_opts_init.restype = None
        L.kevd_kernel_exp.argtypes = [vp, i64, vp, vp]
        L.kevd_kernel_exp.restype = ctypes.c_int
        L.kevd_trace_enable.argtypes = [ctypes.c_int]
        L.kevd_trace_enable.restype = ctypes.c_int
        L.kevd_trace_reset.argtypes = []
        L.kevd_trace_reset.restype = None
        L.kevd_trace_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        L.kevd_trace_read.restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(status):
    return lib().kevd_status_string(int(status)).decode()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _ldf(F):
    """Leading dimension of an (r, N) view whose rows are contiguous: the row stride."""
    if F.dim() != 2 or F.stride(1) != 1 or (F.shape[0] > 1 and F.stride(0) < F.shape[1]):
        raise ValueError("F must be an (r, N) view with contiguous rows")
    return F.stride(0) if F.shape[0] > 1 else F.shape[1]


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _dtype_code(t):
    if t.dtype == torch.float64:
        return KEVD_F64
    if t.dtype == torch.float32:
        return KEVD_F32
    raise TypeError("unsupported dtype %s" % t.dtype)


def make_opts(mode="arpc", b=64, seed=0, until_rank=False, max_rounds=0, precision=KEVD_PREC_FP64, tol=None):
    """Options struct from the library's defaults (kevd_opts_init: tol = 0 for the FP64
    path, 1e-6 for the precision form) with the given fields set."""
    m = {"greedy": KEVD_GREEDY, "arpc": KEVD_ARPC}[mode]
    precision = PRECISIONS.get(precision, precision)
    o = kevd_opts()
    lib().kevd_opts_init(ctypes.byref(o), int(precision))
    o.mode = m
    o.block_b = 1 if m == KEVD_GREEDY else int(b)
    o.until_rank = int(bool(until_rank))
    o.max_rounds = int(max_rounds)
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    if tol is not None:
        o.tol = float(tol)
    return o


def workspace_bytes(which, N, d, r, k=1, opts=None):
    o = ctypes.byref(opts) if opts is not None else None
    return int(lib().kevd_workspace_bytes(which, int(N), int(d), int(r), int(k), o))


def _workspace(nbytes, dev):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)


def _check(call, status):
    if status != KEVD_OK:
        raise KevdError(call, status)


def rpchol_factor(X, eps, r, mode="arpc", b=64, seed=0, until_rank=False, max_rounds=0, F=None,
                  record_proposals=False, precision=None, tol=None):
    """Partial Cholesky factor of the implicit Gaussian kernel matrix of X.

    X: (N, d) CUDA tensor, row-major; float64 selects the FP64 path, float32
    the precision form ("bf16x3": tensor-core split products, FP32 F).
    Returns a dict with F as an (r, N) tensor (the column-major N x r factor;
    F.T is N x r), pivots, rho, rank, rounds, trace_err and, if requested, the
    per-round proposals.
    """
    if precision is None:
        precision = "bf16x3" if X.dtype == torch.float32 else "fp64"
    f_dtype = torch.float32 if PRECISIONS.get(precision, precision) == KEVD_PREC_BF16X3 else torch.float64
    if not X.is_cuda or not X.is_contiguous() or X.dim() != 2:
        raise ValueError("X must be a contiguous 2-D CUDA tensor")
    dev = X.device
    N, d = X.shape
    opts = make_opts(mode, b, seed, until_rank, max_rounds, precision, tol)
    bb = opts.block_b
    if F is None:
        F = torch.empty((r, N), dtype=f_dtype, device=dev)
    piv = torch.empty(r, dtype=torch.int64, device=dev)
    rho = torch.empty(N, dtype=torch.float64, device=dev)
    rounds_max = (max_rounds if max_rounds > 0 else 4 * ((r + bb - 1) // bb) + 16) if until_rank else (
        r if mode == "greedy" else r // bb)
    props = torch.full((max(rounds_max, 1) * bb,), -1, dtype=torch.int64, device=dev) if record_proposals else None
    ws = _workspace(workspace_bytes(KEVD_WS_FACTOR, N, d, r, 1, opts), dev)
    info = kevd_factor_info()
    st = lib().rpchol_factor(_ptr(X), _dtype_code(X), N, d, float(eps), int(r), ctypes.byref(opts), _ptr(F),
                             _dtype_code(F), N, _ptr(piv), _ptr(rho), _ptr(props), ctypes.byref(info), _ptr(ws),
                             ws.numel(), _stream(dev))
    _check("rpchol_factor", st)
    out = dict(F=F, pivots=piv, rho=rho, rank=info.rank, rounds=info.rounds, trace_err=info.trace_err,
               sum_m_sq=info.sum_m_sq, sum_k=info.sum_k, engine_rounds=info.engine_rounds)
    if props is not None:
        out["proposals"] = props.view(-1, bb)[: info.rounds]
    return out


def kernel_exp(t):
    """exp(t) for t <= 0 as the FP64 engine on the tensor cores computes kernel values
    (a CUDA float64 tensor; 0 for t <= -708)."""
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("t must be a contiguous CUDA float64 tensor")
    out = torch.empty_like(t)
    _check("kevd_kernel_exp", lib().kevd_kernel_exp(_ptr(t), t.numel(), _ptr(out), _stream(t.device)))
    return out


def _norm_opts(F):
    """Options that size the normalisation workspace for F's element type."""
    return make_opts("arpc", 64, 0, precision="bf16x3" if F.dtype == torch.float32 else "fp64")


def bistoch_normalize(F, rank):
    """(d~, q~, A, C) from the factor F given as an (r, N) tensor (column-major N x r)."""
    dev = F.device
    N = F.shape[1]
    dtil = torch.empty(N, dtype=torch.float64, device=dev)
    qtil = torch.empty(N, dtype=torch.float64, device=dev)
    A = torch.empty((rank, rank), dtype=torch.float64, device=dev)
    C = torch.empty((rank, rank), dtype=torch.float64, device=dev)
    ws = _workspace(workspace_bytes(KEVD_WS_NORMALIZE, N, 1, rank, 1, _norm_opts(F)), dev)
    st = lib().bistoch_normalize(_ptr(F), _dtype_code(F), N, int(rank), _ldf(F), _ptr(dtil), _ptr(qtil), _ptr(A), _ptr(C),
                                 _ptr(ws), ws.numel(), _stream(dev))
    _check("bistoch_normalize", st)
    return dtil, qtil, A, C


def eig_topk(F, rank, dtil, A, C, k, tau=1e-13):
    """(eigenvalues descending (k,), U as a (k, N) tensor = column-major N x k, kept)."""
    dev = F.device
    N = F.shape[1]
    ev = torch.empty(k, dtype=torch.float64, device=dev)
    U = torch.empty((k, N), dtype=torch.float64, device=dev)
    kept = ctypes.c_int32(0)
    ws = _workspace(workspace_bytes(KEVD_WS_EIG, N, 1, rank, k), dev)
    st = lib().eig_topk(_ptr(F), _dtype_code(F), N, int(rank), _ldf(F), _ptr(dtil), _ptr(A), _ptr(C), int(k), float(tau),
                        _ptr(ev), _ptr(U), ctypes.byref(kept), _ptr(ws), ws.numel(), _stream(dev))
    _check("eig_topk", st)
    return ev, U, kept.value


def symmetric_normalize(F, rank):
    """(d~, A_s = F^T D~^-1 F) from F given as an (r, N) tensor (Section 2.1)."""
    dev = F.device
    N = F.shape[1]
    dtil = torch.empty(N, dtype=torch.float64, device=dev)
    As = torch.empty((rank, rank), dtype=torch.float64, device=dev)
    ws = _workspace(workspace_bytes(KEVD_WS_NORMALIZE, N, 1, rank, 1, _norm_opts(F)), dev)
    _check("symmetric_normalize", lib().symmetric_normalize(_ptr(F), _dtype_code(F), N, int(rank), _ldf(F), _ptr(dtil),
                                                            _ptr(As), _ptr(ws), ws.numel(), _stream(dev)))
    return dtil, As


def symmetric_eig_topk(F, rank, dtil, As, k):
    """Top-k eigenpairs of L~ = D~^-1/2 F F^T D~^-1/2: (eigenvalues (k,), U as a (k, N) tensor)."""
    dev = F.device
    N = F.shape[1]
    ev = torch.empty(k, dtype=torch.float64, device=dev)
    U = torch.empty((k, N), dtype=torch.float64, device=dev)
    ws = _workspace(workspace_bytes(KEVD_WS_EIG, N, 1, rank, k), dev)
    _check("symmetric_eig_topk", lib().symmetric_eig_topk(_ptr(F), _dtype_code(F), N, int(rank), _ldf(F), _ptr(dtil),
                                                          _ptr(As), int(k), _ptr(ev), _ptr(U), _ptr(ws), ws.numel(),
                                                          _stream(dev)))
    return ev, U


def constant_eigvec_fix(U):
    """In place: U(:,0) = 1/sqrt(N), then re-orthonormalise (U given as a (k, N) tensor)."""
    k, N = U.shape
    ws = _workspace(workspace_bytes(KEVD_WS_FIX, N, 0, k, k), U.device)
    _check("constant_eigvec_fix", lib().constant_eigvec_fix(_ptr(U), N, int(k), _ptr(ws), ws.numel(),
                                                            _stream(U.device)))
    return U


def _colmajor(W):
    """(storage tensor, ld) of a matrix view whose columns are contiguous."""
    if W.dim() != 2 or W.stride(0) != 1 or (W.shape[1] > 1 and W.stride(1) < W.shape[0]):
        raise ValueError("W must be a column-major matrix view (e.g. the W returned by rpchol_factor_lowmem)")
    return W, (W.stride(1) if W.shape[1] > 1 else W.shape[0])


def _lowmem_X(X):
    if not X.is_cuda or not X.is_contiguous() or X.dim() != 2 or X.dtype != torch.float64:
        raise ValueError("X must be a contiguous 2-D float64 CUDA tensor")
    return X.shape


def rpchol_factor_lowmem(X, eps, r, mode="arpc", b=64, seed=0, until_rank=False, max_rounds=0,
                         record_proposals=False, tol=None):
    """Low-memory ARPC (FP64): only the pivots S and W = F(S,:) are returned.

    W is an (r, r) column-major view (W[i, j] = F(S_i, j), lower triangular
    on its leading rank x rank block, zero elsewhere); F = K(:,S) W^-T.
    """
    N, d = _lowmem_X(X)
    dev = X.device
    opts = make_opts(mode, b, seed, until_rank, max_rounds, KEVD_PREC_FP64, tol)
    bb = opts.block_b
    Wt = torch.empty((r, r), dtype=torch.float64, device=dev)   # row c of Wt is column c of W
    piv = torch.empty(r, dtype=torch.int64, device=dev)
    rho = torch.empty(N, dtype=torch.float64, device=dev)
    rounds_max = (max_rounds if max_rounds > 0 else 4 * ((r + bb - 1) // bb) + 16) if until_rank else (
        r if mode == "greedy" else r // bb)
    props = torch.full((max(rounds_max, 1) * bb,), -1, dtype=torch.int64, device=dev) if record_proposals else None
    ws = _workspace(workspace_bytes(KEVD_WS_LOWMEM_FACTOR, N, d, r, 1, opts), dev)
    info = kevd_factor_info()
    st = lib().rpchol_factor_lowmem(_ptr(X), N, d, float(eps), int(r), ctypes.byref(opts), _ptr(Wt), r, _ptr(piv),
                                    _ptr(rho), _ptr(props), ctypes.byref(info), _ptr(ws), ws.numel(), _stream(dev))
    _check("rpchol_factor_lowmem", st)
    out = dict(W=Wt.t(), pivots=piv, rho=rho, rank=info.rank, rounds=info.rounds, trace_err=info.trace_err,
               sum_m_sq=info.sum_m_sq, sum_k=info.sum_k, engine_rounds=info.engine_rounds)
    if props is not None:
        out["proposals"] = props.view(-1, bb)[: info.rounds]
    return out


def bistoch_normalize_lowmem(X, eps, pivots, W, rank):
    """(d~, q~, A, C) of the factor F = K(:,S) W^-T, from X, the pivots and W."""
    N, d = _lowmem_X(X)
    dev = X.device
    Wm, ldw = _colmajor(W)
    dtil = torch.empty(N, dtype=torch.float64, device=dev)
    qtil = torch.empty(N, dtype=torch.float64, device=dev)
    A = torch.empty((rank, rank), dtype=torch.float64, device=dev)
    C = torch.empty((rank, rank), dtype=torch.float64, device=dev)
    ws = _workspace(workspace_bytes(KEVD_WS_LOWMEM_NORMALIZE, N, d, rank), dev)
    st = lib().bistoch_normalize_lowmem(_ptr(X), N, d, float(eps), _ptr(pivots), _ptr(Wm), ldw, int(rank), _ptr(dtil),
                                        _ptr(qtil), _ptr(A), _ptr(C), _ptr(ws), ws.numel(), _stream(dev))
    _check("bistoch_normalize_lowmem", st)
    return dtil, qtil, A, C


def eig_topk_lowmem(X, eps, pivots, W, rank, dtil, A, C, k, tau=1e-13):
    """eig_topk for F = K(:,S) W^-T: (eigenvalues descending (k,), U as a (k, N) tensor, kept)."""
    N, d = _lowmem_X(X)
    dev = X.device
    Wm, ldw = _colmajor(W)
    ev = torch.empty(k, dtype=torch.float64, device=dev)
    U = torch.empty((k, N), dtype=torch.float64, device=dev)
    kept = ctypes.c_int32(0)
    ws = _workspace(workspace_bytes(KEVD_WS_LOWMEM_EIG, N, d, rank, k), dev)
    st = lib().eig_topk_lowmem(_ptr(X), N, d, float(eps), _ptr(pivots), _ptr(Wm), ldw, int(rank), _ptr(dtil), _ptr(A),
                               _ptr(C), int(k), float(tau), _ptr(ev), _ptr(U), ctypes.byref(kept), _ptr(ws),
                               ws.numel(), _stream(dev))
    _check("eig_topk_lowmem", st)
    return ev, U, kept.value


def trace_enable(on=True):
    return bool(lib().kevd_trace_enable(int(bool(on))))


def trace_reset():
    lib().kevd_trace_reset()


def trace_read():
    """{stage: (milliseconds, launch groups)} accumulated since the last reset."""
    n = len(STAGES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check("kevd_trace_read", lib().kevd_trace_read(ms, cnt, n))
    return {STAGES[i]: (ms[i], cnt[i]) for i in range(n)}


class Batch:
    """Batched ARPC factorisation of many independent problems (FP64).

    problems: list of dicts with X (CUDA float64, N x d), eps, r, b, seed.
    Outputs per problem (F as an (r, N) tensor, pivots, rho) are allocated
    here; run() replays the captured round loop and returns per-problem info.
    """

    def __init__(self, problems, use_graph=True):
        if not problems:
            raise ValueError("empty batch")
        self.dev = problems[0]["X"].device
        self.out = []
        arr = (kevd_problem * len(problems))()
        for q, p in enumerate(problems):
            X = p["X"]
            if X.dtype != torch.float64 or not X.is_contiguous():
                raise ValueError("batched problems take contiguous float64 X")
            N, d = X.shape
            r = int(p["r"])
            F = torch.empty((r, N), dtype=torch.float64, device=self.dev)
            piv = torch.empty(r, dtype=torch.int64, device=self.dev)
            rho = torch.empty(N, dtype=torch.float64, device=self.dev)
            self.out.append(dict(X=X, F=F, pivots=piv, rho=rho))
            arr[q] = kevd_problem(X.data_ptr(), N, d, r, int(p["b"]), 0, float(p["eps"]),
                                  int(p.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF, F.data_ptr(), N, piv.data_ptr(),
                                  rho.data_ptr())
        self._arr = arr
        nb = int(lib().kevd_batch_workspace_bytes(arr, len(problems)))
        if nb == 0:
            raise KevdError("kevd_batch_workspace_bytes", KEVD_EINVAL)
        self.ws = _workspace(nb, self.dev)
        h = ctypes.c_void_p(0)
        st = lib().kevd_batch_create(arr, len(problems), int(bool(use_graph)), _ptr(self.ws), self.ws.numel(),
                                     _stream(self.dev), ctypes.byref(h))
        _check("kevd_batch_create", st)
        self.h = h

    def run(self):
        n = len(self.out)
        infos = (kevd_factor_info * n)()
        _check("kevd_batch_run", lib().kevd_batch_run(self.h, _stream(self.dev), infos))
        res = []
        for q in range(n):
            o = dict(self.out[q])
            o.update(rank=infos[q].rank, rounds=infos[q].rounds, trace_err=infos[q].trace_err,
                     sum_m_sq=infos[q].sum_m_sq, sum_k=infos[q].sum_k, engine_rounds=infos[q].engine_rounds)
            res.append(o)
        return res

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().kevd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
