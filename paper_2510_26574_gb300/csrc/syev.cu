// Top-k eigenpairs of a dense symmetric r x r matrix (the r x r EVD of
// Section 2 / Algorithm 1, M = R C R^T on the Cholesky route), FP64
// throughout, built for a GPU whose FP64 rate is 1/64 of FP32 and on which
// the library tridiagonal reduction is bound by per-column launch latency.
//
//  1. k_sytrd: Householder tridiagonalisation Q^T M Q = T (the unblocked
//     reduction of LAPACK's sytd2, lower form), one persistent cooperative
//     launch with one grid barrier per column.  Each block keeps the current
//     and previous reflector and w in shared memory and recomputes them
//     redundantly (O(r) per column), every warp owns rows of the trailing
//     matrix (row r in block r mod G) and applies the rank-2 update of column
//     i-1 fused with the symmetric product of column i in a single pass.
//     Reflectors are stored as LAPACK does (below the subdiagonal, tau), so
//     the back-transformation is cuSOLVER's ormtr.
//  2. k_tri_eig: per wanted eigenvalue one block: bisection on Sturm counts
//     (LDL^T pivots with the usual pivmin guard) to full FP64 resolution,
//     then inverse iteration (partial-pivoting LU of T - lambda I, three
//     solves) from a deterministic pseudo-random start.
//  3. CholeskyQR2 of the k vectors in eigenvalue order (Gram-Schmidt
//     semantics: vectors of well separated eigenvalues are left unchanged to
//     rounding, members of a cluster become an orthonormal basis of it).
//  4. cuSOLVER ormtr: V = Q Z.
// Eigenvalues come out ascending (the top k of M), vectors in the same order,
// as the library's subset eigensolver returns them.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "trace.cuh"

namespace kevd {

constexpr int kSyThreads = 512;
constexpr int kSyWarps = kSyThreads / 32;

// Block-wide FP64 sum; every thread gets the same value (fixed order).
__device__ __forceinline__ double sy_block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kSyWarps; ++q) s += red[q];
    __syncthreads();
    return s;
}

// Grid barrier for a cooperative launch (all blocks co-resident).  Bounded:
// gives up after ~1 s or when another block has failed, and reports it.
__device__ bool sy_grid_sync(unsigned* count, unsigned* gen, unsigned& my_gen, int* err) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = my_gen;
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*(volatile unsigned*)gen == g) {
                if (*(volatile int*)err || clock64() - t0 > (1ll << 31)) {
                    ok = 0;
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        my_gen = g + 1;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Copy the upper triangle of a column-major symmetric n x n matrix to its lower one.
__global__ void k_sy_mirror(double* __restrict__ A, int n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);   // A(i, j), column-major
    if (i > j) A[e] = A[(int64_t)i * n + j];
}

// Householder vector of x = [alpha, x2] (LAPACK's dlarfg): beta, tau and the
// scale applied to x2 (v = [1, scale * x2]).
__device__ __forceinline__ void sy_larfg(double alpha, double xnorm2, double& beta, double& tau, double& scale) {
    if (xnorm2 == 0.0) {
        beta = alpha;
        tau = 0.0;
        scale = 1.0;
        return;
    }
    const double nrm = sqrt(alpha * alpha + xnorm2);
    beta = alpha >= 0.0 ? -nrm : nrm;
    tau = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
}

// A: n x n symmetric, full storage (row r of the array = column r).  On exit
// d (n), e (n-1), tau (n-1) and the reflectors below the subdiagonal.
// P: 2 x n (double-buffered symmetric products), bar: {count, gen}, err.
__global__ void __launch_bounds__(kSyThreads) k_sytrd(double* __restrict__ A, int n, double* __restrict__ d,
                                                      double* __restrict__ e, double* __restrict__ tau,
                                                      double* __restrict__ P, unsigned* bar, int* err) {
    extern __shared__ double sy_smem[];
    double* vb0 = sy_smem;          // reflector buffers (indexed by column)
    double* vb1 = sy_smem + n;
    double* wv = sy_smem + 2 * n;   // p, then w
    __shared__ double red[kSyWarps];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int G = gridDim.x, b = blockIdx.x;
    unsigned my_gen = 0;

    // ---- column 0 ----
    double tau_prev = 0.0;
    {
        double part = 0.0;
        for (int c = 1 + tid; c < n; c += kSyThreads) {
            const double x = __ldcg(A + c);
            vb0[c] = x;
            if (c >= 2) part += x * x;
        }
        const double xn2 = sy_block_sum(part, red);
        double beta = 0.0, tv = 0.0, sc = 1.0;
        if (n >= 2) sy_larfg(vb0[1], xn2, beta, tv, sc);
        for (int c = 2 + tid; c < n; c += kSyThreads) vb0[c] *= sc;
        __syncthreads();
        if (tid == 0 && n >= 2) vb0[1] = 1.0;
        if (b == 0 && tid == 0) {
            d[0] = __ldcg(A);
            if (n >= 2) {
                e[0] = beta;
                tau[0] = tv;
            }
        }
        __syncthreads();
        tau_prev = tv;
        if (n >= 2) {
            for (int r = b + G * wid; r < n; r += G * kSyWarps) {
                if (r < 1) continue;
                double s = 0.0;
                for (int c = 1 + lane; c < n; c += 32) s = fma(__ldcg(A + (int64_t)r * n + c), vb0[c], s);
                s = warp_sum(s);
                if (lane == 0) P[r] = tv * s;
            }
            if (!sy_grid_sync(bar, bar + 1, my_gen, err)) return;
        }
    }

    // ---- columns 1 .. n-1 ----
    for (int i = 1; i < n; ++i) {
        double* vp = (i & 1) ? vb0 : vb1;   // reflector i-1 (vp[i] = 1)
        double* vc = (i & 1) ? vb1 : vb0;   // column i, then reflector i
        const double* Pin = P + (int64_t)((i - 1) & 1) * n;
        double* Pout = P + (int64_t)(i & 1) * n;
        // w = p + K v with K = -tau/2 (p . v)
        double part = 0.0;
        for (int r = i + tid; r < n; r += kSyThreads) {
            const double pr = __ldcg(Pin + r);
            wv[r] = pr;
            part += pr * vp[r];
        }
        const double K = -0.5 * tau_prev * sy_block_sum(part, red);
        for (int r = i + tid; r < n; r += kSyThreads) wv[r] = fma(K, vp[r], wv[r]);
        __syncthreads();
        // column i after the rank-2 update of reflector i-1
        const double wi = wv[i];
        part = 0.0;
        for (int c = i + tid; c < n; c += kSyThreads) {
            const double x = __ldcg(A + (int64_t)i * n + c) - (wv[c] + wi * vp[c]);   // vp[i] = 1
            vc[c] = x;
            if (c >= i + 2) part += x * x;
        }
        const double xn2 = sy_block_sum(part, red);
        const double di = vc[i];
        double beta = 0.0, tv = 0.0, sc = 1.0;
        if (i <= n - 2) sy_larfg(vc[i + 1], xn2, beta, tv, sc);
        for (int c = i + 2 + tid; c < n; c += kSyThreads) vc[c] *= sc;
        if (b == 0) {
            // reflector i-1 goes below the subdiagonal of column i-1 (no block reads that row any more)
            for (int c = i + 1 + tid; c < n; c += kSyThreads) A[(int64_t)(i - 1) * n + c] = vp[c];
            if (tid == 0) {
                d[i] = di;
                if (i <= n - 2) {
                    e[i] = beta;
                    tau[i] = tv;
                }
            }
        }
        __syncthreads();
        if (tid == 0 && i <= n - 2) vc[i + 1] = 1.0;
        __syncthreads();
        if (i > n - 2) break;
        // rows r > i: rank-2 update of reflector i-1, fused with the product by reflector i
        for (int r = b + G * wid; r < n; r += G * kSyWarps) {
            if (r <= i) continue;
            const double vr = vp[r], wr = wv[r];
            double* Ar = A + (int64_t)r * n;
            double s = 0.0;
            for (int c = i + 1 + lane; c < n; c += 32) {
                const double a = Ar[c] - (vr * wv[c] + wr * vp[c]);
                Ar[c] = a;
                s = fma(a, vc[c], s);
            }
            s = warp_sum(s);
            if (lane == 0) Pout[r] = tv * s;
        }
        tau_prev = tv;
        if (!sy_grid_sync(bar, bar + 1, my_gen, err)) return;
    }
}

// Number of eigenvalues of T (diagonal dg, squared off-diagonal e2) below x.
__device__ __forceinline__ int sy_sturm(const double* __restrict__ dg, const double* __restrict__ e2, int n, double x,
                                        double pivmin) {
    double q = dg[0] - x;
    int cnt = q < 0.0;
    for (int j = 1; j < n; ++j) {
        if (fabs(q) < pivmin) q = -pivmin;
        q = (dg[j] - x) - e2[j - 1] / q;
        cnt += q < 0.0;
    }
    return cnt;
}

__device__ __forceinline__ double sy_start(uint32_t i, uint32_t j) {   // deterministic start vector entry in [-1, 1)
    uint64_t z = ((uint64_t)j << 32 | i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// One block (thread 0 works) per wanted eigenvalue j = 0..k-1, ascending index
// n-k+j: bisection, then inverse iteration; lam[j], Z(:, j) (column-major, ld n).
// Shared memory: 5 n doubles + n bytes.
__global__ void k_tri_eig(const double* __restrict__ dg, const double* __restrict__ eo, int n, int k,
                          double* __restrict__ lam, double* __restrict__ Z) {
    extern __shared__ double te_smem[];
    if (threadIdx.x != 0) return;
    const int j = blockIdx.x;
    double* ua = te_smem;          // U diagonal
    double* ub = ua + n;           // U first superdiagonal
    double* uc = ub + n;           // U second superdiagonal
    double* ml = uc + n;           // multipliers
    double* x = ml + n;            // iterate
    unsigned char* pv = reinterpret_cast<unsigned char*>(x + n);
    double* e2 = ub;               // squared off-diagonal, reused before the factorisation
    double tnorm = 0.0, gl = DBL_MAX, gu = -DBL_MAX, emax2 = 0.0;
    for (int i = 0; i < n; ++i) {
        const double ea = i > 0 ? fabs(eo[i - 1]) : 0.0, eb = i < n - 1 ? fabs(eo[i]) : 0.0;
        gl = fmin(gl, dg[i] - ea - eb);
        gu = fmax(gu, dg[i] + ea + eb);
        tnorm = fmax(tnorm, fabs(dg[i]) + ea + eb);
        if (i < n - 1) {
            e2[i] = eo[i] * eo[i];
            emax2 = fmax(emax2, e2[i]);
        }
    }
    const double pivmin = DBL_MIN * fmax(1.0, emax2);
    const int m = n - k + j;   // ascending index of the wanted eigenvalue
    double lo = gl - 2.0 * DBL_EPSILON * tnorm - pivmin, hi = gu + 2.0 * DBL_EPSILON * tnorm + pivmin;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 2.0 * pivmin || mid <= lo || mid >= hi) break;
        if (sy_sturm(dg, e2, n, mid, pivmin) > m) hi = mid;
        else lo = mid;
    }
    const double lmb = 0.5 * (lo + hi);
    lam[j] = lmb;

    // LU with partial pivoting of T - lmb I (LAPACK's dlagtf); tiny pivots -> +-tol
    const double tol = DBL_EPSILON * fmax(tnorm, DBL_MIN);
    for (int i = 0; i < n; ++i) {
        ua[i] = dg[i] - lmb;
        ub[i] = i < n - 1 ? eo[i] : 0.0;
        uc[i] = 0.0;
    }
    for (int i = 0; i < n - 1; ++i) {
        const double cdn = eo[i];   // (i+1, i)
        if (fabs(ua[i]) >= fabs(cdn)) {
            pv[i] = 0;
            const double mult = ua[i] != 0.0 ? cdn / ua[i] : 0.0;
            ml[i] = mult;
            ua[i + 1] -= mult * ub[i];
        } else {
            pv[i] = 1;
            const double mult = ua[i] / cdn;
            ml[i] = mult;
            ua[i] = cdn;
            const double t = ua[i + 1];
            ua[i + 1] = ub[i] - mult * t;
            if (i < n - 2) {
                uc[i] = ub[i + 1];
                ub[i + 1] = -mult * ub[i + 1];
            }
            ub[i] = t;
        }
    }
    for (int i = 0; i < n; ++i)
        if (fabs(ua[i]) < tol) ua[i] = ua[i] < 0.0 ? -tol : tol;

    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
        x[i] = sy_start((uint32_t)i, (uint32_t)m);
        nrm += x[i] * x[i];
    }
    for (int sweep = 0; sweep < 3; ++sweep) {
        const double s0 = 1.0 / sqrt(nrm);
        for (int i = 0; i < n; ++i) x[i] *= s0;
        // forward: apply the row interchanges and multipliers
        for (int i = 0; i < n - 1; ++i) {
            if (pv[i]) {
                const double t = x[i];
                x[i] = x[i + 1];
                x[i + 1] = t - ml[i] * x[i + 1];
            } else {
                x[i + 1] -= ml[i] * x[i];
            }
        }
        // backward: U y = x
        x[n - 1] /= ua[n - 1];
        if (n >= 2) x[n - 2] = (x[n - 2] - ub[n - 2] * x[n - 1]) / ua[n - 2];
        for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - ub[i] * x[i + 1] - uc[i] * x[i + 2]) / ua[i];
        nrm = 0.0;
        double amax = 0.0;
        for (int i = 0; i < n; ++i) amax = fmax(amax, fabs(x[i]));
        const double sa = amax > 0.0 ? 1.0 / amax : 1.0;   // guard the squares against overflow
        for (int i = 0; i < n; ++i) {
            x[i] *= sa;
            nrm += x[i] * x[i];
        }
    }
    const double s1 = 1.0 / sqrt(nrm);
    for (int i = 0; i < n; ++i) Z[(int64_t)j * n + i] = x[i] * s1;
}

}  // namespace kevd

using namespace kevd;

// Doubles of workspace the native solver needs beyond the caller's M, lam, Z
// and the solver work array: P (2n), d, e, tau (3n), the barrier words, the
// k x k Gram and its split partials.
size_t kevd_gram_partial_doubles(int64_t N, int k);
cudaError_t kevd_gram_plain(const double* U, int64_t ldu, int64_t N, int k, double* G, double* gpart, cudaStream_t s);

size_t kevd_syev_ws_doubles(int n, int k) {
    return (size_t)5 * n + 16 + (size_t)k * k + kevd_gram_partial_doubles(n, k);
}

// Largest n the native solver takes (shared memory of k_sytrd and k_tri_eig).
int kevd_syev_max_n() { return 5000; }

// Top-k eigenpairs of the symmetric n x n matrix M (column-major, upper
// triangle read, destroyed): lam[0..k-1] ascending, Z (n x k, ld n) the
// orthonormal eigenvectors in the same order.  ws: kevd_syev_ws_doubles
// doubles; work / lwork: cuSOLVER work for potrf(k) and ormtr(n, k); info:
// 2 ints.  Returns a KEVD status.
int kevd_syev_topk(cusolverDnHandle_t h, cublasHandle_t hb, double* M, int n, int k, double* lam, double* Z,
                   double* ws, double* work, int lwork, int* info, cudaStream_t s) {
    if (n < 1 || k < 1 || k > n || n > kevd_syev_max_n()) return KEVD_EINVAL;
    double* P = ws;
    double* dg = P + 2 * n;
    double* eo = dg + n;
    double* tau = eo + n;
    unsigned* bar = reinterpret_cast<unsigned*>(tau + n);
    int* err = reinterpret_cast<int*>(bar + 2);
    double* G = tau + n + 16;
    double* gpart = G + (size_t)k * k;

    int dev = 0, nsm = 0, occ = 0;
    KEVD_CUDA_TRY(cudaGetDevice(&dev));
    KEVD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t sm1 = (size_t)3 * n * sizeof(double);
    KEVD_CUDA_TRY(cudaFuncSetAttribute(k_sytrd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    KEVD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sytrd, kSyThreads, sm1));
    if (occ < 1) return KEVD_ECUDA;
    const int grid = std::max(1, std::min(nsm * occ, (n + 7) / 8));
    {
        TraceScope tr(kStSolver, s);
        k_sy_mirror<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(M, n);
        KEVD_CUDA_TRY(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s));
        int nn = n;
        void* args[] = {&M, &nn, &dg, &eo, &tau, &P, &bar, &err};
        KEVD_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_sytrd, dim3(grid), dim3(kSyThreads), args, sm1, s));
        const size_t sm2 = (size_t)5 * n * sizeof(double) + n;
        KEVD_CUDA_TRY(cudaFuncSetAttribute(k_tri_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
        k_tri_eig<<<k, 32, sm2, s>>>(dg, eo, n, k, lam, Z);
        KEVD_CUDA_TRY(cudaGetLastError());
        // CholeskyQR2 of Z in eigenvalue order
        const double one = 1.0;
        if (cublasSetStream(hb, s) != CUBLAS_STATUS_SUCCESS) return KEVD_ECUDA;
        for (int pass = 0; pass < 2; ++pass) {
            KEVD_CUDA_TRY(kevd_gram_plain(Z, n, n, k, G, gpart, s));
            if (cusolverDnDpotrf(h, CUBLAS_FILL_MODE_UPPER, k, G, k, work, lwork, info) != CUSOLVER_STATUS_SUCCESS)
                return KEVD_ECUDA;
            if (cublasDtrsm(hb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, n, k, &one,
                            G, k, Z, n) != CUBLAS_STATUS_SUCCESS)
                return KEVD_ECUDA;
        }
        // V = Q Z
        if (n >= 2 && cusolverDnDormtr(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, n, k, M, n, tau, Z, n,
                                       work, lwork, info + 1) != CUSOLVER_STATUS_SUCCESS)
            return KEVD_ECUDA;
    }
    int herr = 0, hinfo[2] = {0, 0};
    KEVD_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaMemcpyAsync(hinfo, info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr) return KEVD_ETIMEOUT;
    if (hinfo[0] != 0 || hinfo[1] != 0) return KEVD_EEIG;
    return KEVD_OK;
}
