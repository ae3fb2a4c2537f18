// Low-memory ARPC (Appendix A, closing paragraph; Remark of Section 4.2), FP64:
// rpchol_factor_lowmem, bistoch_normalize_lowmem and the lift of
// eig_topk_lowmem.
//
// Only the accepted pivots S and W = F(S,:) (rank x rank, lower triangular:
// the Cholesky factor of K(S,S)) are kept.  Every row of F is
// F(i,:) = K(i,S) W^-T, so no N x r array exists: the N-long passes work on a
// row panel of P rows (P x r doubles, at most 128 MiB) of kernel values
// K(panel, S) = exp(-(|x_i|^2 + |x_s|^2 - 2 x_i.x_s) / eps), formed by a DGEMM
// of the panel's rows of X against X(S,:) and an exp kernel.
//
// rpchol_factor_lowmem, one round of Algorithm 2 with k pivots so far:
//   a2  proposals from rho (the FP64 path's kernel);
//   a3  F(S',:) = K(S',S) W^-T (b x k kernel block, then a triangular solve),
//       H = K(S',S') - F(S',:) F(S',:)^T (the FP64 path's kernel);
//   a4  Algorithm 3 (the FP64 path's kernel): accepted T, L = chol(H(T,T));
//   W   gains the rows [F(T,:) | L]; Z = W^-T F(T,:)^T (k x m);
//   a5  per panel R = K(p,T) - K(p,S) Z (= K(p,T) - F(p,:) F(T,:)^T),
//       G = R L^-T, rho -= rownorms(G)^2 clamped at 0, tile statistics.
// The host reads (k, m) once per round to size the library calls.
//
// bistoch_normalize_lowmem, three passes over the panels:
//   1  s_K = K(S,:) 1                       y = W^-T W^-1 s_K  (so F s = K(:,S) y)
//   2  d~ = K(:,S) y,  t_K = K(S,:) d~^-1   z = W^-T W^-1 t_K
//   3  q~ = K(:,S) z;  F_p = K(p,S) W^-T;  A += F_p^T D~^-2 F_p,
//      C += F_p^T Q~^-1 F_p (the normalisation's Gram kernel, accumulated).
// The vectors come from K(:,S) times a solved vector, which agrees with the
// rebuilt-F definition to ~1e-14 even at cond(W) ~ 3e5.  The Grams use the
// rebuilt F_p: W^-1 (K^T D K) W^-T loses accuracy with cond(W)^2 (2e-10 at
// cond(W) = 6e3).
//
// The lift of eig_topk_lowmem: U = D~^-1 K(:,S) (W^-T Y), per panel.
//
// DGEMM, DGEMV and the triangular solves are cuBLAS calls (plain library
// products); set-up, exp, residual update, statistics and Grams are kernels of
// this library.
#include <cublas_v2.h>

#include <algorithm>
#include <climits>
#include <cstdlib>

#include "common.cuh"
#include "factor.cuh"
#include "lowmem.cuh"
#include "trace.cuh"

cudaError_t kevd_gram_weighted(const double* F, int64_t ldf, int64_t N, int rank, const double* wa, const double* wc,
                               double* gpart, double* A, double* C, int acc, cudaStream_t s);
size_t kevd_gram_partial_doubles(int64_t N, int k);

#define LM_BLAS(expr)                                               \
    do {                                                            \
        if ((expr) != CUBLAS_STATUS_SUCCESS) return KEVD_ECUDA;     \
    } while (0)

namespace kevd {

// cuBLAS handle per device and host thread, bound to stream s.
static cublasHandle_t lm_blas(cudaStream_t s) {
    thread_local cublasHandle_t handles[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!handles[dev] && cublasCreate(&handles[dev]) != CUBLAS_STATUS_SUCCESS) handles[dev] = nullptr;
    if (!handles[dev] || cublasSetStream(handles[dev], s) != CUBLAS_STATUS_SUCCESS) return nullptr;
    return handles[dev];
}

constexpr size_t kLmPanelDoubles = size_t(1) << 24;   // 128 MiB of kernel values per panel

// Rows per panel: a multiple of the 64-row rho tile, at most 2^24 / r (at
// least 64), and no more than N rounded up to the tile.  KEVD_LOWMEM_PANEL=rows
// in the environment lowers the 2^24 / r rule (rounded down to a multiple of
// 64, at least 64; a larger value is capped by the rule, so P r stays within
// 2^24 doubles and every panel index fits an int); workspace sizing and the
// calls must see the same setting.
static int64_t lm_panel_rows(int64_t N, int r) {
    int64_t p = (int64_t)(kLmPanelDoubles / (size_t)std::max(r, 1));
    if (const char* e = getenv("KEVD_LOWMEM_PANEL")) {
        const long long v = atoll(e);
        if (v > 0 && v < p) p = v;
    }
    p = std::max<int64_t>(p / kBM * kBM, kBM);
    return std::min<int64_t>(p, (N + kBM - 1) / kBM * kBM);
}

// A panel of kernel values and the pivot rows it is formed from.
struct LmPanel {
    double* xn;    // N: |x_i|^2
    double* XS;    // r x d row-major: X(S,:)
    double* xnS;   // r: |x_s|^2
    double* Kp;    // P x r column-major (ld P)
    int64_t P;
};

// own_xn = false: |x_i|^2 lives elsewhere (the caller sets p.xn).
static LmPanel carve_panel(Carver& c, int64_t N, int d, int r, bool own_xn = true) {
    LmPanel p;
    p.P = lm_panel_rows(N, r);
    p.xn = own_xn ? c.take<double>(N) : nullptr;
    p.XS = c.take<double>((size_t)r * d);
    p.xnS = c.take<double>(r);
    p.Kp = c.take<double>((size_t)p.P * r);
    return p;
}

// |x_i|^2, summed in the order of the FP64 path's set-up kernel.
__global__ void k_lm_norms(const double* __restrict__ X, int64_t N, int d, double* __restrict__ xn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* x = X + i * d;
    double s = 0.0;
    for (int c = 0; c < d; ++c) s = fma(x[c], x[c], s);
    xn[i] = s;
}

// XS(a,:) = X(S_a,:) and xnS(a) = |x_{S_a}|^2 for a < n.  A pivot outside
// [0, N) sets flags bit 2 and is not read.
__global__ void k_lm_gather(const double* __restrict__ X, int64_t N, int d, const int64_t* __restrict__ piv, int n,
                            const double* __restrict__ xn, double* __restrict__ XS, double* __restrict__ xnS,
                            int* __restrict__ flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * d) return;
    const int a = (int)(e / d), c = (int)(e % d);
    const int64_t p = piv[a];
    if (p < 0 || p >= N) {
        if (c == 0) atomicOr(flags, 4);
        XS[e] = 0.0;
        if (c == 0) xnS[a] = 0.0;
        return;
    }
    XS[e] = X[p * d + c];
    if (c == 0) xnS[a] = xn[p];
}

// Kernel values over the DGEMM's dot products, in place:
// Kp(i,a) = exp(-max(|x_i|^2 + |x_s|^2 - 2 Kp(i,a), 0) / eps) with i the row
// i0 + i and s = S_a (exactly 1 where the row is the pivot itself), divided by
// rowdiv(i0 + i) when rowdiv is given.
__global__ void k_lm_kexp(double* __restrict__ Kp, int64_t P, int64_t Pc, int n, int64_t i0,
                          const double* __restrict__ xn, const double* __restrict__ xnS,
                          const int64_t* __restrict__ piv, double inv_eps, const double* __restrict__ rowdiv) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Pc * n) return;
    const int64_t i = e % Pc;
    const int a = (int)(e / Pc);
    const int64_t row = i0 + i;
    double* kp = Kp + (int64_t)a * P + i;
    double v;
    if (piv[a] == row) v = 1.0;
    else v = exp(-fmax(xn[row] + xnS[a] - 2.0 * *kp, 0.0) * inv_eps);
    if (rowdiv) v /= rowdiv[row];
    *kp = v;
}

// Kp(0:Pc, 0:n) = K(i0:i0+Pc, S_0:S_n) [/ rowdiv]: one DGEMM of the panel's
// rows of X against X(S,:), then the exp kernel.
static int kernel_panel(cublasHandle_t h, const double* X, int d, int64_t i0, int64_t Pc, int n, const LmPanel& p,
                        const int64_t* piv, double inv_eps, const double* rowdiv, cudaStream_t s) {
    const double one = 1.0, zero = 0.0;
    LM_BLAS(cublasDgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)Pc, n, d, &one, X + i0 * d, d, p.XS, d, &zero, p.Kp,
                        (int)p.P));
    const int64_t tot = Pc * n;
    k_lm_kexp<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(p.Kp, p.P, Pc, n, i0, p.xn, p.xnS, piv, inv_eps, rowdiv);
    KEVD_LAUNCH_CHECK();
    return KEVD_OK;
}

// ---------------------------------------------------------------------------
// Factor kernels
// ---------------------------------------------------------------------------

// X(S',:) of the proposals as a d x b panel (XSP) and their |x|^2 (xnS): the
// FP64 path's gather without the rows of F.
__global__ void k_lm_gather_prop(FactorWs w, const double* __restrict__ X, int d, int b) {
    if (w.st->done) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d * b) return;
    const int j = e % b, c = e / b;
    const int64_t p = w.prop[j];
    w.XSP[(size_t)c * b + j] = X[p * d + c];
    if (c == 0) w.xnS[j] = w.xn[p];
}

// K(S', S) of the b proposals against the k pivots, column-major b x k (ld b),
// into FSP (a triangular solve with W then turns it into F(S',:)).
__global__ void k_lm_kq(FactorWs w, const double* __restrict__ XS, const double* __restrict__ xnS,
                        const int64_t* __restrict__ piv, int k, int d, int b, double inv_eps) {
    if (w.st->done) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * k) return;
    const int j = e % b, a = e / b;
    double dot = 0.0;
    for (int c = 0; c < d; ++c) dot = fma(w.XSP[(size_t)c * b + j], XS[(size_t)a * d + c], dot);
    double v;
    if (w.prop[j] == piv[a]) v = 1.0;
    else v = exp(-fmax(w.xnS[j] + xnS[a] - 2.0 * dot, 0.0) * inv_eps);
    w.FSP[(size_t)a * b + j] = v;
}

// Rows k..k+m-1 of W = [F(T,:k) | L], Zt = F(T,:k)^T (k x m, ld k), and the
// new pivots' rows of XS and entries of xnS.  One thread per (a, column).
__global__ void k_lm_extend(FactorWs w, const double* __restrict__ X, int d, int k, int m, int b,
                            const int64_t* __restrict__ piv, double* __restrict__ W, int64_t ldw,
                            double* __restrict__ XS, double* __restrict__ xnS, double* __restrict__ Zt) {
    const int width = k + m + d;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * width) return;
    const int a = (int)(e / width), c = (int)(e % width);
    if (c < k) {
        const double v = w.FSP[(size_t)c * b + w.acc_pos[a]];
        W[(int64_t)c * ldw + k + a] = v;
        Zt[(size_t)a * k + c] = v;
    } else if (c < k + m) {
        const int a2 = c - k;
        W[(int64_t)(k + a2) * ldw + k + a] = a2 <= a ? w.Lc[(size_t)a * b + a2] : 0.0;
    } else {
        const int cc = c - k - m;
        const int64_t p = piv[k + a];
        XS[(size_t)(k + a) * d + cc] = X[p * d + cc];
        if (cc == 0) xnS[k + a] = w.xn[p];
    }
}

// rho -= rownorms(G)^2 (G = R L^-T, P-strided columns), clamped at 0, and the
// per-64-row-tile sum and (max, lowest index) of rho that the proposal kernel
// reads, summed in the FP64 engine's order.  256 threads = 4 tiles; i0 is a
// multiple of 64.
__global__ void __launch_bounds__(256) k_lm_rho(FactorWs w, const double* __restrict__ G, int64_t P, int64_t Pc,
                                                int m, int64_t i0, double* __restrict__ rho) {
    __shared__ double ssum[8], smax[8];
    __shared__ int64_t sidx[8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t li = (int64_t)blockIdx.x * 256 + tid;
    double rnew = 0.0, rmax = -1.0;
    int64_t ridx = LLONG_MAX;
    if (li < Pc) {
        const int64_t row = i0 + li;
        double nrm = 0.0;
        for (int j = 0; j < m; ++j) {
            const double g = G[(int64_t)j * P + li];
            nrm = fma(g, g, nrm);
        }
        rnew = fmax(rho[row] - nrm, 0.0);
        rho[row] = rnew;
        rmax = rnew;
        ridx = row;
    }
    const double sw = warp_sum(rnew);
    warp_argmax(rmax, ridx);
    if (lane == 0) {
        ssum[wid] = sw;
        smax[wid] = rmax;
        sidx[wid] = ridx;
    }
    __syncthreads();
    if (tid < 4) {
        const int64_t lt = (int64_t)blockIdx.x * 256 + 64 * tid;   // first local row of the tile
        if (lt < Pc) {
            double ts = 0.0, tm = -1.0;
            int64_t ti = LLONG_MAX;
            for (int q = 2 * tid; q < 2 * tid + 2; ++q) {
                ts += ssum[q];
                argmax_merge(tm, ti, smax[q], sidx[q]);
            }
            const int64_t t = (i0 + lt) / kBM;
            w.tile_sum[t] = ts;
            w.tile_max[t] = tm;
            w.tile_idx[t] = ti;
        }
    }
}

// ---------------------------------------------------------------------------
// Normalisation kernels
// ---------------------------------------------------------------------------
__global__ void k_lm_fill(double* __restrict__ x, int64_t n, double v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// 1/d~ of a panel's rows; flags bit 0 where d~ <= 0 (Algorithm 1, first assert).
__global__ void k_lm_recip(const double* __restrict__ d, int64_t n, double* __restrict__ out, int* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!(d[i] > 0.0)) atomicOr(flags, 1);
    out[i] = 1.0 / d[i];
}

// Gram weights 1/d~^2 and 1/q~ of a panel's rows; flags bit 1 where q~ <= 0.
__global__ void k_lm_weights(const double* __restrict__ d, const double* __restrict__ q, int64_t n,
                             double* __restrict__ wa, double* __restrict__ wc, int* __restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!(q[i] > 0.0)) atomicOr(flags, 2);
    wa[i] = 1.0 / (d[i] * d[i]);
    wc[i] = 1.0 / q[i];
}

static int grid1(int64_t n) { return (int)((n + 255) / 256); }

// ---------------------------------------------------------------------------
// Workspaces
// ---------------------------------------------------------------------------
struct LmFactorWs {
    FactorWs w;
    LmPanel p;
    double* Zt;    // r x b: F(T,:)^T, then W^-T F(T,:)^T
};

static LmFactorWs carve_lm_factor(void* base, int64_t N, int d, int r, int b, size_t* bytes) {
    LmFactorWs L;
    size_t fb = 0;
    L.w = carve_factor_fp64(base, N, d, r, b, &fb);
    Carver c(base);
    c.off = fb;
    L.p = carve_panel(c, N, d, r, false);
    L.p.xn = L.w.xn;   // |x_i|^2 of the FP64 path's workspace
    L.Zt = c.take<double>((size_t)r * b);
    *bytes = c.off;
    return L;
}

struct LmNormWs {
    LmPanel p;
    double* ones;   // P
    double* vec;    // rank: K(S,:) 1, then K(S,:) d~^-1
    double* y;      // rank: the solved vectors
    double* pv;     // P: 1/d~ of the panel's rows
    double* wa;     // P: 1/d~^2
    double* wc;     // P: 1/q~
    double* gpart;  // Gram split partials of one panel
    int* flags;     // bit 0: d~ <= 0, bit 1: q~ <= 0, bit 2: pivot out of range
};

static LmNormWs carve_lm_norm(void* base, int64_t N, int d, int rank, size_t* bytes) {
    Carver c(base);
    LmNormWs L;
    L.p = carve_panel(c, N, d, rank);
    const int64_t P = L.p.P;
    L.ones = c.take<double>(P);
    L.vec = c.take<double>(rank);
    L.y = c.take<double>(rank);
    L.pv = c.take<double>(P);
    L.wa = c.take<double>(P);
    L.wc = c.take<double>(P);
    L.gpart = c.take<double>(kevd_gram_partial_doubles(P, rank));
    L.flags = c.take<int>(4);
    *bytes = c.off;
    return L;
}

static int lm_rounds(const kevd_opts* o, int r, int b, int greedy) {
    if (o->until_rank) return o->max_rounds > 0 ? o->max_rounds : 4 * ((r + b - 1) / b) + 16;
    return greedy ? r : r / b;
}

static bool aligned(const void* p) { return reinterpret_cast<uintptr_t>(p) % kAlign == 0; }

// y := W^-T W^-1 y (two triangular solves with the lower triangular W).
static int solve_ww(cublasHandle_t h, const double* W, int64_t ldw, int rank, double* y) {
    LM_BLAS(cublasDtrsv(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, rank, W, (int)ldw, y, 1));
    LM_BLAS(cublasDtrsv(h, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, rank, W, (int)ldw, y, 1));
    return KEVD_OK;
}

}  // namespace kevd

using namespace kevd;

size_t kevd_lowmem_factor_ws(int64_t N, int32_t d, int32_t r, const kevd_opts* o) {
    if (!o || N < 1 || d < 1 || r < 1 || r > N) return 0;
    const int b = o->mode == KEVD_GREEDY ? 1 : o->block_b;
    if (b < 1 || b > 128) return 0;
    size_t bytes = 0;
    carve_lm_factor(nullptr, N, d, r, b, &bytes);
    return bytes;
}

size_t kevd_lowmem_normalize_ws(int64_t N, int32_t d, int32_t rank) {
    if (N < 1 || d < 1 || rank < 1 || rank > N) return 0;
    size_t bytes = 0;
    carve_lm_norm(nullptr, N, d, rank, &bytes);
    return bytes;
}

size_t kevd_lowmem_lift_bytes(int64_t N, int d, int rank) {
    Carver c(nullptr);
    carve_panel(c, N, d, rank);
    c.take<int>(4);
    return c.off;
}

extern "C" int rpchol_factor_lowmem(const double* X, int64_t N, int32_t d, double eps, int32_t r,
                                    const kevd_opts* opts, double* W, int64_t ldw, int64_t* pivots, double* rho,
                                    int64_t* proposals, kevd_factor_info* info, void* workspace, size_t ws_bytes,
                                    void* stream) {
    if (!opts || !X || !W || !pivots || !rho || !info) return KEVD_EINVAL;
    if (N < 1 || N > INT_MAX || d < 1 || r < 1 || r > N || ldw < r || ldw > INT_MAX) return KEVD_EINVAL;
    if (!(eps > 0.0) || !isfinite(eps)) return KEVD_EINVAL;
    if (opts->mode != KEVD_GREEDY && opts->mode != KEVD_ARPC) return KEVD_EINVAL;
    if (opts->precision != KEVD_PREC_FP64) return KEVD_EINVAL;
    if (opts->reserved != 0 || opts->max_rounds < 0) return KEVD_EINVAL;
    if (!(opts->tol >= 0.0 && opts->tol < 1.0)) return KEVD_EINVAL;
    const int greedy = opts->mode == KEVD_GREEDY;
    const int b = greedy ? 1 : opts->block_b;
    if (b < 1 || b > 128) return KEVD_EINVAL;
    const int rounds = lm_rounds(opts, r, b, greedy);
    if (rounds < 1) return KEVD_EINVAL;
    size_t need = 0;
    LmFactorWs L = carve_lm_factor(workspace, N, d, r, b, &need);
    if (!workspace || ws_bytes < need || !aligned(workspace)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cublasHandle_t h = lm_blas(s);
    if (!h) return KEVD_ECUDA;
    const FactorWs& w = L.w;
    const LmPanel& p = L.p;
    const double inv_eps = 1.0 / eps, one = 1.0, mone = -1.0;
    {
        TraceScope tr(kStOther, s);
        KEVD_CUDA_TRY(cudaMemset2DAsync(W, (size_t)ldw * sizeof(double), 0, (size_t)r * sizeof(double), r, s));
        launch_prepare_fp64(X, N, d, w, rho, s);
    }
    KEVD_LAUNCH_CHECK();

    int k = 0;   // committed rank, as the proposal kernel will see it
    for (int rnd = 0; rnd < rounds; ++rnd) {
        {
            TraceScope tr(kStPropose, s);
            launch_propose(w, rho, N, b, r, greedy, opts->seed, rnd, proposals, opts->tol * N, s);
        }
        {
            TraceScope tr(kStGather, s);
            k_lm_gather_prop<<<grid1((int64_t)d * b), 256, 0, s>>>(w, X, d, b);
            if (k > 0) {
                k_lm_kq<<<grid1((int64_t)b * k), 256, 0, s>>>(w, p.XS, p.xnS, pivots, k, d, b, inv_eps);
                LM_BLAS(cublasDtrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, b,
                                    k, &one, W, (int)ldw, w.FSP, b));   // F(S',:) = K(S',S) W^-T
            }
        }
        KEVD_LAUNCH_CHECK();
        {
            TraceScope tr(kStBlockH, s);
            launch_blockH(w, d, b, inv_eps, s);
        }
        {
            TraceScope tr(kStReject, s);
            KEVD_CUDA_TRY(launch_reject(w, b, r, greedy, opts->seed, rnd, pivots, s));
        }
        FactorState hs;
        KEVD_CUDA_TRY(cudaMemcpyAsync(&hs, w.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        KEVD_CUDA_TRY(cudaStreamSynchronize(s));
        if (hs.done) break;
        if (hs.k != k) return KEVD_ECUDA;
        const int m = hs.m;
        if (m == 0) continue;
        TraceScope tr(kStEngine, s);
        k_lm_extend<<<grid1((int64_t)m * (k + m + d)), 256, 0, s>>>(w, X, d, k, m, b, pivots, W, ldw, p.XS, p.xnS,
                                                                   L.Zt);
        KEVD_LAUNCH_CHECK();
        if (k > 0)   // Z = W^-T F(T,:)^T with the leading k x k block of W
            LM_BLAS(cublasDtrsm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, k, m,
                                &one, W, (int)ldw, L.Zt, k));
        for (int64_t i0 = 0; i0 < N; i0 += p.P) {
            const int64_t Pc = std::min(p.P, N - i0);
            const int st = kernel_panel(h, X, d, i0, Pc, k + m, p, pivots, inv_eps, nullptr, s);
            if (st != KEVD_OK) return st;
            double* R = p.Kp + (int64_t)k * p.P;
            if (k > 0)   // R = K(p,T) - K(p,S) Z
                LM_BLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)Pc, m, k, &mone, p.Kp, (int)p.P, L.Zt, k, &one,
                                    R, (int)p.P));
            // G = R L^-T: Lc is L row-major (ld b), i.e. L^T column-major
            LM_BLAS(cublasDtrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, (int)Pc,
                                m, &one, w.Lc, b, R, (int)p.P));
            k_lm_rho<<<grid1(Pc), 256, 0, s>>>(w, R, p.P, Pc, m, i0, rho);
            KEVD_LAUNCH_CHECK();
        }
        k += m;
    }
    {
        TraceScope tr(kStOther, s);
        launch_finalize(w, rho, N, s);
    }
    KEVD_LAUNCH_CHECK();
    FactorState hs;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&hs, w.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    info->rank = hs.k;
    info->rounds = hs.rounds;
    info->trace_err = hs.final_sum;
    info->sum_m_sq = hs.sum_m_sq;
    info->sum_k = hs.sum_k;
    info->engine_rounds = hs.eng_rounds;
    if (hs.bad) return KEVD_EINVAL;
    return KEVD_OK;
}

extern "C" int bistoch_normalize_lowmem(const double* X, int64_t N, int32_t d, double eps, const int64_t* pivots,
                                        const double* W, int64_t ldw, int32_t rank, double* dtil, double* qtil,
                                        double* A, double* C, void* workspace, size_t ws_bytes, void* stream) {
    if (!X || !pivots || !W || !dtil || !qtil || !A || !C) return KEVD_EINVAL;
    if (N < 1 || N > INT_MAX || d < 1 || rank < 1 || rank > N || ldw < rank || ldw > INT_MAX) return KEVD_EINVAL;
    if (!(eps > 0.0) || !isfinite(eps)) return KEVD_EINVAL;
    size_t need = 0;
    LmNormWs L = carve_lm_norm(workspace, N, d, rank, &need);
    if (!workspace || ws_bytes < need || !aligned(workspace)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cublasHandle_t h = lm_blas(s);
    if (!h) return KEVD_ECUDA;
    const LmPanel& p = L.p;
    const double inv_eps = 1.0 / eps, one = 1.0, zero = 0.0;
    const bool one_panel = N <= p.P;   // the panel is formed once and kept for all three passes
    int st;

    KEVD_CUDA_TRY(cudaMemsetAsync(L.flags, 0, 4 * sizeof(int), s));
    {
        TraceScope tr(kStDegree, s);
        k_lm_norms<<<grid1(N), 256, 0, s>>>(X, N, d, p.xn);
        k_lm_gather<<<grid1((int64_t)rank * d), 256, 0, s>>>(X, N, d, pivots, rank, p.xn, p.XS, p.xnS, L.flags);
        k_lm_fill<<<grid1(p.P), 256, 0, s>>>(L.ones, p.P, 1.0);
        KEVD_LAUNCH_CHECK();
        // pass 1: K(S,:) 1, then y = W^-T W^-1 K(S,:) 1
        KEVD_CUDA_TRY(cudaMemsetAsync(L.vec, 0, (size_t)rank * sizeof(double), s));
        for (int64_t i0 = 0; i0 < N; i0 += p.P) {
            const int64_t Pc = std::min(p.P, N - i0);
            if ((st = kernel_panel(h, X, d, i0, Pc, rank, p, pivots, inv_eps, nullptr, s)) != KEVD_OK) return st;
            LM_BLAS(cublasDgemv(h, CUBLAS_OP_T, (int)Pc, rank, &one, p.Kp, (int)p.P, L.ones, 1, &one, L.vec, 1));
        }
        KEVD_CUDA_TRY(cudaMemcpyAsync(L.y, L.vec, (size_t)rank * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if ((st = solve_ww(h, W, ldw, rank, L.y)) != KEVD_OK) return st;
        // pass 2: d~ = K(:,S) y and K(S,:) d~^-1, then y = W^-T W^-1 K(S,:) d~^-1
        KEVD_CUDA_TRY(cudaMemsetAsync(L.vec, 0, (size_t)rank * sizeof(double), s));
        for (int64_t i0 = 0; i0 < N; i0 += p.P) {
            const int64_t Pc = std::min(p.P, N - i0);
            if (!one_panel &&
                (st = kernel_panel(h, X, d, i0, Pc, rank, p, pivots, inv_eps, nullptr, s)) != KEVD_OK)
                return st;
            LM_BLAS(cublasDgemv(h, CUBLAS_OP_N, (int)Pc, rank, &one, p.Kp, (int)p.P, L.y, 1, &zero, dtil + i0, 1));
            k_lm_recip<<<grid1(Pc), 256, 0, s>>>(dtil + i0, Pc, L.pv, L.flags);
            KEVD_LAUNCH_CHECK();
            LM_BLAS(cublasDgemv(h, CUBLAS_OP_T, (int)Pc, rank, &one, p.Kp, (int)p.P, L.pv, 1, &one, L.vec, 1));
        }
        KEVD_CUDA_TRY(cudaMemcpyAsync(L.y, L.vec, (size_t)rank * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if ((st = solve_ww(h, W, ldw, rank, L.y)) != KEVD_OK) return st;
    }
    {
        // pass 3: q~ = K(:,S) y; F_p = K(p,S) W^-T; A += F_p^T D~^-2 F_p, C += F_p^T Q~^-1 F_p
        TraceScope tr(kStGram, s);
        for (int64_t i0 = 0; i0 < N; i0 += p.P) {
            const int64_t Pc = std::min(p.P, N - i0);
            if (!one_panel &&
                (st = kernel_panel(h, X, d, i0, Pc, rank, p, pivots, inv_eps, nullptr, s)) != KEVD_OK)
                return st;
            LM_BLAS(cublasDgemv(h, CUBLAS_OP_N, (int)Pc, rank, &one, p.Kp, (int)p.P, L.y, 1, &zero, qtil + i0, 1));
            k_lm_weights<<<grid1(Pc), 256, 0, s>>>(dtil + i0, qtil + i0, Pc, L.wa, L.wc, L.flags);
            KEVD_LAUNCH_CHECK();
            LM_BLAS(cublasDtrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, (int)Pc,
                                rank, &one, W, (int)ldw, p.Kp, (int)p.P));
            KEVD_CUDA_TRY(kevd_gram_weighted(p.Kp, p.P, Pc, rank, L.wa, L.wc, L.gpart, A, C, i0 > 0, s));
        }
    }
    int flags = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&flags, L.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    if (flags & 4) return KEVD_EINVAL;
    if (flags & 1) return KEVD_ED_NONPOS;
    if (flags & 2) return KEVD_EQ_NONPOS;
    return KEVD_OK;
}

int kevd_lowmem_lift(const KevdLowmemLift& Lf, int64_t N, int rank, int k, double* Y, const double* dtil, double* U,
                     cudaStream_t s) {
    Carver c(Lf.ws);
    const LmPanel p = carve_panel(c, N, Lf.d, rank);
    int* flags = c.take<int>(4);
    cublasHandle_t h = lm_blas(s);
    if (!h) return KEVD_ECUDA;
    const double one = 1.0, zero = 0.0;
    int st;
    {
        TraceScope tr(kStLift, s);
        KEVD_CUDA_TRY(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
        LM_BLAS(cublasDtrsm(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, CUBLAS_DIAG_NON_UNIT, rank, k, &one,
                            Lf.W, (int)Lf.ldw, Y, rank));   // Y := W^-T Y
        k_lm_norms<<<grid1(N), 256, 0, s>>>(Lf.X, N, Lf.d, p.xn);
        k_lm_gather<<<grid1((int64_t)rank * Lf.d), 256, 0, s>>>(Lf.X, N, Lf.d, Lf.piv, rank, p.xn, p.XS, p.xnS, flags);
        KEVD_LAUNCH_CHECK();
        for (int64_t i0 = 0; i0 < N; i0 += p.P) {   // U(p,:) = D~^-1 K(p,S) (W^-T Y)
            const int64_t Pc = std::min(p.P, N - i0);
            if ((st = kernel_panel(h, Lf.X, Lf.d, i0, Pc, rank, p, Lf.piv, Lf.inv_eps, dtil, s)) != KEVD_OK) return st;
            LM_BLAS(cublasDgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)Pc, k, rank, &one, p.Kp, (int)p.P, Y, rank, &zero,
                                U + i0, (int)N));
        }
    }
    int hf = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    return (hf & 4) ? KEVD_EINVAL : KEVD_OK;
}
