// eig_topk: top-k eigenpairs of P~ = B C B^T with B = D~^-1 F (Section 2, the
// B C B^T method; Section 2.2; Algorithm 1 lines for the QR, the r x r EVD and
// U = Q1 V), FP64 path, all device-resident.
//
// Range basis of B from the Gram A = B^T B instead of a Householder QR of the
// N x r matrix B:
//  * Cholesky route (used when A is numerically positive definite):
//      A = R^T R (R upper), Q1 = B R^-1, M = R C R^T, top-k of M = V Lambda V^T,
//      U = Q1 V_k = D~^-1 F Y with Y = R^-1 V_k.
//  * Spectral route (fallback when the Cholesky factorisation breaks down):
//      A = W S W^T, Q1 = B W S^-1/2 on the directions with S_j > tau max S (the
//      others get weight 0, which replaces the paper's gamma regularisation of
//      the QR), M = S^1/2 W^T C W S^1/2, Y = W S^-1/2 V_k.
// The lift is one N x r x k GEMM with the row scaling by 1/d~ in its epilogue.
// Factorisations and eigensolves of the r x r matrices call cuSOLVER (potrf,
// syevdx for the top k, syevd) and the back substitution Y = R^-1 V_k calls
// cuBLAS trsm; every other step is a kernel of this file (R C and the upper
// half of (R C) R^T skip the zero triangles of R).  On this GPU the tridiagonal reduction inside syevd dominates (24 ms
// at r = 800), so the Cholesky route saves one full eigensolve.
#include <cublas_v2.h>
#include <cusolverDn.h>

#include <algorithm>
#include <type_traits>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "lowmem.cuh"
#include "oz_digits.cuh"
#include "ozgemm.cuh"
#include "trace.cuh"

size_t kevd_gram_partial_doubles(int64_t N, int k);
cudaError_t kevd_gram_plain(const double* U, int64_t ldu, int64_t N, int k, double* G, double* gpart, cudaStream_t s);

// Native top-k symmetric eigensolver (syev.cu).
size_t kevd_syev_ws_doubles(int n, int k);
int kevd_syev_max_n();
int kevd_syev_topk(cusolverDnHandle_t h, cublasHandle_t hb, double* M, int n, int k, double* lam, double* Z,
                   double* ws, double* work, int lwork, int* info, cudaStream_t s);

namespace kevd {

// The r x r top-k eigensolve calls cuSOLVER's syevdx.  KEVD_SYEV=native in the
// environment selects the library's own tridiagonalisation and tridiagonal
// solver (syev.cu) for r up to kevd_syev_max_n().  It matches syevdx to the FP64
// bars but is slower on this GPU: its one-column-per-barrier reduction costs
// what cuSOLVER's sytrd costs (~20 us per column), and its bisection is a chain
// of dependent FP64 operations, each ~130 cycles here.
static bool use_native_syev(int r) {
    const char* v = getenv("KEVD_SYEV");
    return v && std::strcmp(v, "native") == 0 && r <= kevd_syev_max_n();
}

// ---------------------------------------------------------------------------
// cuSOLVER handle per device and host thread (created on first use, kept until
// exit): a handle carries its stream, so threads that drive different streams
// concurrently each need their own.
// ---------------------------------------------------------------------------
static cusolverDnHandle_t solver_handle() {
    thread_local cusolverDnHandle_t handles[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!handles[dev] && cusolverDnCreate(&handles[dev]) != CUSOLVER_STATUS_SUCCESS) handles[dev] = nullptr;
    return handles[dev];
}

// cuBLAS handle per device and host thread (triangular solve of the r x k back-substitution).
static cublasHandle_t blas_handle() {
    thread_local cublasHandle_t handles[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!handles[dev] && cublasCreate(&handles[dev]) != CUBLAS_STATUS_SUCCESS) handles[dev] = nullptr;
    return handles[dev];
}

// Doubles of device workspace for the largest of the r x r solver calls.
static int subspace_b(int r, int k);

static int64_t solver_lwork(int n, int k, size_t* trtri_host) {
    cusolverDnHandle_t h = solver_handle();
    if (!h) return -1;
    int l1 = 0, l2 = 0, l3 = 0, meig = 0;
    if (cusolverDnDsyevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, nullptr, n,
                                    nullptr, &l1) != CUSOLVER_STATUS_SUCCESS)
        return -1;
    if (cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_UPPER, n, nullptr, n, &l2) != CUSOLVER_STATUS_SUCCESS)
        return -1;
    if (cusolverDnDsyevdx_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER, n,
                                     nullptr, n, 0.0, 0.0, n - k + 1, n, &meig, nullptr, &l3) != CUSOLVER_STATUS_SUCCESS)
        return -1;
    size_t td = 0, th = 0;
    if (cusolverDnXtrtri_bufferSize(h, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, n, CUDA_R_64F, nullptr, n, &td,
                                    &th) != CUSOLVER_STATUS_SUCCESS)
        return -1;
    if (trtri_host) *trtri_host = th;
    int l4 = 0;
    if (n >= 2 && cusolverDnDormtr_bufferSize(h, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, n, k, nullptr, n,
                                              nullptr, nullptr, n, &l4) != CUSOLVER_STATUS_SUCCESS)
        return -1;
    int l5 = 0, l6 = 0;   // Householder QR of the subspace solver's first block (r x b)
    const int b = subspace_b(n, k);
    if (b > 0 && (cusolverDnDgeqrf_bufferSize(h, n, b, nullptr, n, &l5) != CUSOLVER_STATUS_SUCCESS ||
                  cusolverDnDorgqr_bufferSize(h, n, b, b, nullptr, n, nullptr, &l6) != CUSOLVER_STATUS_SUCCESS))
        return -1;
    return std::max<int64_t>({l1, l2, l3, (int64_t)((td + 7) / 8), l4, l5, l6});
}

// Block size of the precision form's subspace top-k solver (0: not used): b =
// 2k + 32 columns, taken when b <= r/3.  Its cost is seven b-column
// orthonormalisations plus one b x b eigensolve (latency-bound library calls:
// ~3.5 ms and ~17 ms at b = 544), against the subset eigensolver's reduction of
// the whole r x r matrix (~73 ms at r = 1,848).
static int subspace_b(int r, int k) {
    const int b = 2 * k + 32;
    return b <= r / 3 ? b : 0;
}

// G, B (b x b each), theta (b), Z (r x k), residual ratios (k), Householder scalars (b).
static size_t subspace_ws_doubles(int r, int k) {
    const int b = subspace_b(r, k);
    if (b == 0) return 1;
    return (size_t)2 * b * b + 2 * b + (size_t)r * k + k;
}

// FP32 lift tiling (k_lift32 below)
constexpr int kLT = 128;   // output tile (n and j)
constexpr int kLK = 16;    // columns of F per chunk
constexpr int kLS = 4;     // pipeline stages
static inline int lift_rp(int r) { return (r + kLK - 1) / kLK * kLK; }
static inline int lift_kp(int k) { return (k + kLT - 1) / kLT * kLT; }

struct EigWs {
    double* W;      // r x r: A, then its eigenvectors
    double* S;      // r: eigenvalues of A (ascending)
    double* sh;     // r: sqrt(S_j) or 0
    double* sih;    // r: 1/sqrt(S_j) or 0
    double* Z;      // r x r: W diag(sh)
    double* CZ;     // r x r
    double* M;      // r x r: M, then its eigenvectors
    double* lam;    // r
    double* Vt;     // r x k: diag(sih) V_k
    double* Y;      // r x k
    double* work;   // lwork
    int* info;      // 2 solver infos + kept count
    double* cmax;   // k: signed entry of largest magnitude per column
    int64_t* cidx;  // k
    double* rowdiv; // N: sqrt(d~) for the symmetric lift
    double* sy;     // native eigensolver workspace
    double* ss;     // subspace top-k workspace (precision form)
    float* Yt;      // rp x kp: FP32 k-major copy of Y for the FP32 lift
    double* frow;   // N: max_c |F(i, c)| (FP64 lift on the tensor cores)
    double* Yp;     // k x ldyp: Y^T, rows padded to an even length
    double* ymax;   // k: max_c |Y(c, j)|
    int* ozflag;    // bit 2: a bounded wait of the tensor-core lift gave up
    uint16_t* lp;   // digit planes of one row slab of F (lift from planes, ozmm.cu); before the
                    // lift, the planes of the r x r stage's operands (at least 14 r ldk)
    uint16_t* yp;   // digit planes of Y^T: 7 x k x ldk
    int* fexp;      // row exponents of the slab
    int* ye;        // k: row exponents of Y^T
    int* rre;       // 3 r: row exponents of the r x r stage's planes
};

static inline int lift_ldyp(int r) { return (r + 1) / 2 * 2; }

// Lift from digit planes: F is cut into K-major planes (row-contiguous K = r, padded
// to 16) one row slab at a time, within kLiftPlaneBudget bytes.
constexpr size_t kLiftPlaneBudget = (size_t)2 << 30;
static inline int lift_ldk(int r) { return (r + 15) / 16 * 16; }
static inline int64_t lift_slab(int64_t N, int r, int D) {
    int64_t S = (int64_t)(kLiftPlaneBudget / ((size_t)2 * D * lift_ldk(r))) / 128 * 128;
    S = std::max<int64_t>(S, 128);
    return std::min<int64_t>(S, (N + 127) / 128 * 128);
}

static EigWs carve_eig(void* base, int64_t N, int r, int k, int64_t lwork, size_t* bytes) {
    Carver c(base);
    EigWs w;
    const size_t rr = (size_t)r * r;
    w.W = c.take<double>(rr);
    w.S = c.take<double>(r);
    w.sh = c.take<double>(r);
    w.sih = c.take<double>(r);
    w.Z = c.take<double>(rr);
    w.CZ = c.take<double>(rr);
    w.M = c.take<double>(rr);
    w.lam = c.take<double>(r);
    w.Vt = c.take<double>((size_t)r * k);
    w.Y = c.take<double>((size_t)r * k);
    w.work = c.take<double>((size_t)std::max<int64_t>(lwork, 1));
    w.info = c.take<int>(4);
    w.cmax = c.take<double>(k);
    w.cidx = c.take<int64_t>(k);
    w.rowdiv = c.take<double>(N);
    w.sy = c.take<double>(kevd_syev_ws_doubles(r, k));
    w.ss = c.take<double>(subspace_ws_doubles(r, k));
    w.Yt = c.take<float>((size_t)lift_rp(r) * lift_kp(k));
    w.frow = c.take<double>(N);
    w.Yp = c.take<double>((size_t)k * lift_ldyp(r));
    w.ymax = c.take<double>(k);
    w.ozflag = c.take<int>(4);
    const int ldk = lift_ldk(r);
    w.lp = c.take<uint16_t>(std::max({(size_t)3 * lift_slab(N, r, 3), (size_t)kDigits * lift_slab(N, r, kDigits),
                                      (size_t)2 * kDigits * r}) *
                            ldk);
    w.yp = c.take<uint16_t>((size_t)kDigits * k * ldk);
    w.fexp = c.take<int>((size_t)lift_slab(N, r, 3));
    w.ye = c.take<int>(k);
    w.rre = c.take<int>((size_t)3 * r);
    *bytes = c.off;
    return w;
}



// ---------------------------------------------------------------------------
// Column-major FP64 GEMM: C(MxN) = op(A)(MxK) op(B)(KxN), optionally each row
// divided by rowdiv[i].  64 x 64 tiles, 16-deep chunks, 4 x 4 per thread.
// ---------------------------------------------------------------------------
// TAe: element type of A; Acc: arithmetic (double, or float for FP32 F).
template <bool TA, typename TAe, typename Acc>
__global__ void __launch_bounds__(256) k_dgemm(int64_t M, int64_t Nc, int64_t K, const TAe* __restrict__ A,
                                               int64_t lda, const double* __restrict__ B, int64_t ldb,
                                               double* __restrict__ C, int64_t ldc,
                                               const double* __restrict__ rowdiv) {
    using Acc2 = typename std::conditional<std::is_same<Acc, double>::value, double2, float2>::type;
    constexpr int T = 64, BK = 16, P = T + 4;
    __shared__ __align__(16) Acc As[BK][P];
    __shared__ __align__(16) Acc Bs[BK][P];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * T, j0 = (int64_t)blockIdx.y * T;
    Acc acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = Acc(0);
    for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int p = 0; p < (T * BK) / 256; ++p) {
            const int e = tid + 256 * p;
            int i, kk;
            if (TA) { kk = e % BK; i = e / BK; } else { i = e % T; kk = e / T; }
            const int64_t gi = i0 + i, gk = k0 + kk;
            Acc v = Acc(0);
            if (gi < M && gk < K) v = (Acc)(TA ? A[gi * lda + gk] : A[gk * lda + gi]);
            As[kk][i] = v;
        }
#pragma unroll
        for (int p = 0; p < (T * BK) / 256; ++p) {
            const int e = tid + 256 * p, kk = e % BK, j = e / BK;
            const int64_t gj = j0 + j, gk = k0 + kk;
            Bs[kk][j] = (gj < Nc && gk < K) ? (Acc)B[gj * ldb + gk] : Acc(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const Acc2 a0 = *reinterpret_cast<const Acc2*>(&As[kk][ty * 4]);
            const Acc2 a1 = *reinterpret_cast<const Acc2*>(&As[kk][ty * 4 + 2]);
            const Acc2 b0 = *reinterpret_cast<const Acc2*>(&Bs[kk][tx * 4]);
            const Acc2 b1 = *reinterpret_cast<const Acc2*>(&Bs[kk][tx * 4 + 2]);
            const Acc a4[4] = {a0.x, a0.y, a1.x, a1.y}, b4[4] = {b0.x, b0.y, b1.x, b1.y};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = fma(a4[a], b4[c], acc[a][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gi = i0 + ty * 4 + a;
        if (gi >= M) continue;
        const double dv = rowdiv ? rowdiv[gi] : 1.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t gj = j0 + tx * 4 + c;
            if (gj < Nc) C[gj * ldc + gi] = rowdiv ? (double)acc[a][c] / dv : (double)acc[a][c];
        }
    }
}

static void dgemm(bool ta, int64_t M, int64_t Nc, int64_t K, const double* A, int64_t lda, const double* B,
                  int64_t ldb, double* C, int64_t ldc, const double* rowdiv, cudaStream_t s) {
    const dim3 g((unsigned)((M + 63) / 64), (unsigned)((Nc + 63) / 64));
    if (ta) k_dgemm<true, double, double><<<g, 256, 0, s>>>(M, Nc, K, A, lda, B, ldb, C, ldc, rowdiv);
    else k_dgemm<false, double, double><<<g, 256, 0, s>>>(M, Nc, K, A, lda, B, ldb, C, ldc, rowdiv);
}

// ---------------------------------------------------------------------------
// Row maxima of |F(i, :r)| (F column-major); one thread per row, coalesced over rows.
__global__ void k_rowmax_cm(const double* __restrict__ F, int64_t ldf, int64_t N, int r, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double mx = 0.0;
    for (int c = 0; c < r; ++c) mx = fmax(mx, fabs(F[(int64_t)c * ldf + i]));
    out[i] = mx;
}

// Yp(j, c) = Y(c, j) for c < r (zero up to the padded length) and its row maxima;
// block j, Y column-major r x k.
__global__ void k_lift_panel(const double* __restrict__ Y, int r, int ldyp, double* __restrict__ Yp,
                             double* __restrict__ ymax) {
    const int j = blockIdx.x;
    double mx = 0.0;
    for (int c = threadIdx.x; c < ldyp; c += blockDim.x) {
        const double v = c < r ? Y[(int64_t)j * r + c] : 0.0;
        Yp[(int64_t)j * ldyp + c] = v;
        mx = fmax(mx, fabs(v));
    }
    __shared__ double red[32];
#pragma unroll
    for (int q = 16; q; q >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, q));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mx = fmax(mx, red[q]);
        ymax[j] = mx;
    }
}

static bool oz_lift_enabled(const double* F, int64_t ldf, int64_t N) {
    const char* e = getenv("KEVD_LIFT");
    if (e && e[0] == 'f') return false;                       // KEVD_LIFT=fp64: the FP64-pipe GEMM
    return N < ((int64_t)1 << 31) && ozgemm_layout_ok(F, ldf);
}

// Row maxima of |F(i, :r)| (F column-major, FP64 or FP32) as doubles; the FP64
// maximum compares the bits of |x| as integers (FP64 is the slow pipe).
template <typename T>
__global__ void k_rowmax_any(const T* __restrict__ F, int64_t ldf, int64_t N, int r, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if constexpr (std::is_same<T, double>::value) {
        unsigned long long mx = 0;
        for (int c = 0; c < r; ++c)
            mx = max(mx, (unsigned long long)__double_as_longlong(F[(int64_t)c * ldf + i]) & 0x7FFFFFFFFFFFFFFFull);
        out[i] = __longlong_as_double((long long)mx);
    } else {
        float mx = 0.f;
        for (int c = 0; c < r; ++c) mx = fmaxf(mx, fabsf(F[(int64_t)c * ldf + i]));
        out[i] = (double)mx;
    }
}

// D-digit planes of rows [row0, row0 + rows) of F (column-major N x r) with one
// exponent per row from frow: word (s S + il) ldk / 2 + c / 2 holds columns c, c + 1
// of slab row il (zero past r), fexp[il] the row's exponent.  Block: a 32-row x
// 64-column tile transposed through shared memory (reads coalesced down columns,
// plane writes coalesced along rows).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_lift_planes(const T* __restrict__ F, int64_t ldf, int64_t N, int r, int ldk,
                                                     int64_t row0, int rows, int S, const double* __restrict__ frow,
                                                     uint32_t* __restrict__ P, int* __restrict__ fexp) {
    __shared__ T tile[64][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int c0 = blockIdx.x * 64, il0 = blockIdx.y * 32;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = c0 + wid + 8 * j, il = il0 + lane;
        T v = T(0);
        if (c < r && il < rows && row0 + il < N) v = F[(int64_t)c * ldf + row0 + il];
        tile[wid + 8 * j][lane] = v;
    }
    __syncthreads();
    const size_t plane = (size_t)S * (ldk / 2);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int rr = wid + 8 * q, il = il0 + rr;
        if (il >= rows) break;
        const int E = row0 + il < N ? exp_of(frow[row0 + il]) : -900;
        if (blockIdx.x == 0 && lane == 0) fexp[il] = E;
        const int c = c0 + 2 * lane;
        if (c >= ldk) continue;
        long long T0, T1;
        if constexpr (std::is_same<T, double>::value) {
            T0 = oz_T_f64<D>(tile[2 * lane][rr], E);
            T1 = oz_T_f64<D>(tile[2 * lane + 1][rr], E);
        } else {
            T0 = oz_T_f32<D>(tile[2 * lane][rr], E);
            T1 = oz_T_f32<D>(tile[2 * lane + 1][rr], E);
        }
        uint32_t wd[D];
        oz_planes2<D>(T0, T1, wd);
#pragma unroll
        for (int s2 = 0; s2 < D; ++s2) P[s2 * plane + (size_t)il * (ldk / 2) + c / 2] = wd[s2];
    }
}

// D-digit planes of Y^T (row j = column j of Y, r x k column-major; zero past r)
// and their row exponents; one block per row.
template <int D>
__global__ void __launch_bounds__(256) k_lift_ypl(const double* __restrict__ Y, int r, int k, int ldk,
                                                  uint32_t* __restrict__ P, int* __restrict__ ye) {
    const int j = blockIdx.x;
    const double* y = Y + (int64_t)j * r;
    unsigned long long mx = 0;
    for (int c = threadIdx.x; c < r; c += blockDim.x)
        mx = max(mx, (unsigned long long)__double_as_longlong(y[c]) & 0x7FFFFFFFFFFFFFFFull);
    __shared__ unsigned long long red[8];
#pragma unroll
    for (int q = 16; q; q >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, q));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) mx = max(mx, red[q]);
    const int E = exp_of(__longlong_as_double((long long)mx));
    if (threadIdx.x == 0) ye[j] = E;
    const size_t plane = (size_t)k * (ldk / 2);
    for (int c = 2 * threadIdx.x; c < ldk; c += 2 * blockDim.x) {
        uint32_t wd[D];
        oz_planes2<D>(oz_T_f64<D>(c < r ? y[c] : 0.0, E), oz_T_f64<D>(c + 1 < r ? y[c + 1] : 0.0, E), wd);
#pragma unroll
        for (int s2 = 0; s2 < D; ++s2) P[s2 * plane + (size_t)j * (ldk / 2) + c / 2] = wd[s2];
    }
}

// U = diag(1/rowdiv) F Y on the tensor cores from digit planes (D = 7 for FP64 F,
// 3 for FP32 F): per row slab, cut F's rows once (k_lift_planes) and run the
// persistent plane product (k_ozmm) over them.
template <typename T, int D>
static cudaError_t lift_planes(int64_t N, int k, int r, const T* F, int64_t ldf, const double* Y, double* U,
                               const double* rowdiv, const EigWs& w, cudaStream_t s) {
    const int ldk = lift_ldk(r);
    const int64_t S = lift_slab(N, r, D);
    cudaError_t e;
    k_rowmax_any<T><<<(unsigned)((N + 255) / 256), 256, 0, s>>>(F, ldf, N, r, w.frow);
    k_lift_ypl<D><<<k, 256, 0, s>>>(Y, r, k, ldk, reinterpret_cast<uint32_t*>(w.yp), w.ye);
    CUtensorMap ma, mb;
    if (!ozmm_map(&ma, w.lp, S, ldk, S * ldk, true, D) || !ozmm_map(&mb, w.yp, k, ldk, (int64_t)k * ldk, false, D))
        return cudaErrorInvalidValue;
    for (int64_t row0 = 0; row0 < N; row0 += S) {
        const int rows = (int)std::min<int64_t>(S, N - row0);
        k_lift_planes<T, D><<<dim3((unsigned)((ldk + 63) / 64), (unsigned)((rows + 31) / 32)), 256, 0, s>>>(
            F, ldf, N, r, ldk, row0, rows, (int)S, w.frow, reinterpret_cast<uint32_t*>(w.lp), w.fexp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_ozmm(ma, mb, w.fexp, 0, w.ye, 0, rows, k, ldk, nullptr, U + row0, N, 0, nullptr, 0, 0,
                             w.ozflag, s, D, rowdiv ? rowdiv + row0 : nullptr)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// The lift's variant: KEVD_LIFT=fp64 the FP64-pipe GEMM (FP64 F), KEVD_LIFT=slice
// the per-tile slicing product (FP64 F), KEVD_LIFT=ffma the FFMA kernel (FP32 F);
// by default the products from planes.
static char lift_mode() {
    const char* e = getenv("KEVD_LIFT");
    return e && e[0] ? e[0] : 'p';
}

// U = diag(1/rowdiv) F Y with FP64 F: the FP64-accurate tensor-core product
// (ozgemm.cu) when F's layout allows, else the FP64-pipe GEMM.
static cudaError_t lift_fp64(int64_t N, int k, int r, const double* F, int64_t ldf, const double* Y, double* U,
                             const double* rowdiv, const EigWs& w, cudaStream_t s) {
    if (!oz_lift_enabled(F, ldf, N)) {
        dgemm(false, N, k, r, F, ldf, Y, r, U, N, rowdiv, s);
        return cudaGetLastError();
    }
    if (lift_mode() != 's') return lift_planes<double, kDigits>(N, k, r, F, ldf, Y, U, rowdiv, w, s);
    const int ldyp = lift_ldyp(r);
    k_rowmax_cm<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(F, ldf, N, r, w.frow);
    k_lift_panel<<<k, 256, 0, s>>>(Y, r, ldyp, w.Yp, w.ymax);
    return launch_ozgemm(F, ldf, true, N, w.frow, w.Yp, ldyp, k, w.ymax, r, r, nullptr, U, N, rowdiv, w.ozflag, s);
}

// Lift with FP32 F (precision form): U = diag(1/rowdiv) F Y, FFMA products with
// FP32 accumulation over r, FP64 output.  F is column-major N x r, so a chunk
// of 16 columns of one 128-row block is 16 contiguous 512-byte runs, already
// in the k-major layout the micro-tiles read: it is copied to shared memory
// unchanged by 16-byte cp.async (4-byte copies when F or ldf is not 16-byte
// aligned), with zero fill past N and past r.  Y is converted once to an FP32
// k-major copy Yt (rp x kp, zero padded), copied the same way.  Four stages,
// 128 x 128 output tile per 256 threads, 8 x 8 accumulators per thread, with
// the n index on tx so that the FP64 stores of U are contiguous along n.
// ---------------------------------------------------------------------------

__global__ void k_lift_prep(const double* __restrict__ Y, int r, int k, int rp, int kp, float* __restrict__ Yt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rp * kp) return;
    const int l = (int)(e / kp), j = (int)(e % kp);
    Yt[e] = (l < r && j < k) ? (float)Y[(int64_t)j * r + l] : 0.f;
}

__device__ __forceinline__ void lift_cp16(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void lift_cp4(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(256, 1) k_lift32(const float* __restrict__ F, int64_t ldf, int64_t N, int r, int rp,
                                                   const float* __restrict__ Yt, int kp, int k,
                                                   const double* __restrict__ rowdiv, double* __restrict__ U,
                                                   int64_t ldu, int vec) {
    constexpr int kPlane = kLK * kLT;   // floats per operand per stage
    extern __shared__ float4 lift_smem[];
    float* sm = reinterpret_cast<float*>(lift_smem);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t n0 = (int64_t)blockIdx.x * kLT;
    const int j0 = blockIdx.y * kLT;
    const int nch = rp / kLK;

    auto issue = [&](int ch) {
        const int st = ch % kLS;
        const int l0 = ch * kLK;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int e = tid + 256 * p, l = e >> 5, q = e & 31;
            const uint32_t da = sbase + (uint32_t)((st * 2 * kPlane + l * kLT + 4 * q) * 4);
            const uint32_t db = da + (uint32_t)(kPlane * 4);
            const int64_t n = n0 + 4 * q;
            const int64_t left = N - n;
            const bool ok = l0 + l < r && left > 0;
            const float* src = ok ? F + (int64_t)(l0 + l) * ldf + n : F;
            if (vec) {
                lift_cp16(da, src, ok ? (uint32_t)(4 * (left < 4 ? left : 4)) : 0u);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const bool in = ok && t < left;
                    lift_cp4(da + 4 * t, in ? src + t : F, in ? 4u : 0u);
                }
            }
            lift_cp16(db, Yt + (int64_t)(l0 + l) * kp + j0 + 4 * q, 16u);
        }
    };

    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;

#pragma unroll
    for (int ch = 0; ch < kLS - 1; ++ch) {
        if (ch < nch) issue(ch);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int ch = 0; ch < nch; ++ch) {
        asm volatile("cp.async.wait_group %0;" ::"n"(kLS - 2) : "memory");   // chunk ch landed
        __syncthreads();   // ... for every thread; and stage (ch-1) % kLS is no longer read
        if (ch + kLS - 1 < nch) issue(ch + kLS - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        const float* a_s = sm + (ch % kLS) * 2 * kPlane;
        const float* b_s = a_s + kPlane;
#pragma unroll
        for (int kk = 0; kk < kLK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(a_s + kk * kLT + 4 * tx);
            const float4 a1 = *reinterpret_cast<const float4*>(a_s + kk * kLT + 64 + 4 * tx);
            const float4 b0 = *reinterpret_cast<const float4*>(b_s + kk * kLT + 4 * ty);
            const float4 b1 = *reinterpret_cast<const float4*>(b_s + kk * kLT + 64 + 4 * ty);
            const float a8[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(a8[a], b8[c], acc[a][c]);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");

    const bool pair = (ldu % 2 == 0);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t nb = n0 + 64 * h + 4 * tx;   // rows nb .. nb+3 (a = 4h .. 4h+3)
        double dv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) dv[t] = nb + t < N ? rowdiv[nb + t] : 1.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int j = j0 + (c < 4 ? 0 : 64) + 4 * ty + (c & 3);
            if (j >= k) continue;
            double o[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) o[t] = (double)acc[4 * h + t][c] / dv[t];
            double* dst = U + (int64_t)j * ldu + nb;
            if (pair && nb + 4 <= N) {
                reinterpret_cast<double2*>(dst)[0] = make_double2(o[0], o[1]);
                reinterpret_cast<double2*>(dst)[1] = make_double2(o[2], o[3]);
            } else {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (nb + t < N) dst[t] = o[t];
            }
        }
    }
}


static cudaError_t sgemm_lift(int64_t N, int k, int r, const float* F, int64_t ldf, const double* Y, double* U,
                              int64_t ldu, const double* rowdiv, float* Yt, cudaStream_t s) {
    const int rp = lift_rp(r), kp = lift_kp(k);
    k_lift_prep<<<(unsigned)(((int64_t)rp * kp + 255) / 256), 256, 0, s>>>(Y, r, k, rp, kp, Yt);
    const int vec = (reinterpret_cast<uintptr_t>(F) % 16 == 0) && (ldf % 4 == 0);
    const int smem = kLS * 2 * kLK * kLT * (int)sizeof(float);   // 64 KB: above the default 48 KB limit
    const cudaError_t e = cudaFuncSetAttribute(k_lift32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((N + kLT - 1) / kLT), (unsigned)(kp / kLT));
    k_lift32<<<g, 256, smem, s>>>(F, ldf, N, r, rp, Yt, kp, k, rowdiv, U, ldu, vec);
    return cudaGetLastError();
}

// U = diag(1/rowdiv) F Y with FP32 F: three-digit products from planes on the
// tensor cores (FP32-accurate), or the FFMA kernel under KEVD_LIFT=ffma.
static cudaError_t lift_fp32(int64_t N, int k, int r, const float* F, int64_t ldf, const double* Y, double* U,
                             const double* rowdiv, const EigWs& w, cudaStream_t s) {
    if (lift_mode() == 'f' || N >= ((int64_t)1 << 31))
        return sgemm_lift(N, k, r, F, ldf, Y, U, N, rowdiv, w.Yt, s);
    return lift_planes<float, 3>(N, k, r, F, ldf, Y, U, rowdiv, w, s);
}

// ---------------------------------------------------------------------------
// Precision form: top-k eigenpairs of the r x r matrix M by block subspace
// iteration with Rayleigh-Ritz (b = 2k + 32 columns, six power steps after
// Q = orth(M Omega) from a graded start block, CholeskyQR orthonormalisation
// (Householder QR for M Omega when its Gram is numerically singular), syevd of the b x b projection, more
// steps when the check fails and the observed rate allows).  The r x r x b and b x b x r products run FP64-accurate on the
// tensor cores (k_ozmm from seven-digit planes).  Every returned pair is
// checked: |M v - theta v| <= 1e-6 theta bounds each eigenvalue's relative
// error by 1e-6 (Bauer-Fike for symmetric M), far inside the 1e-4 of that
// form; if a pair fails, the caller falls back to the full subset eigensolver.
// M is read only.
// ---------------------------------------------------------------------------
// Start block Omega (r x b, column-major): the first b coordinate vectors plus
// 1e-3 times uniform noise on [-1, 1] (splitmix64 of the entry index).  M is
// graded: its rows and columns follow the pivot order of the partial Cholesky
// factor, whose diagonal decays, so the leading coordinates carry its dominant
// directions.  From coordinate vectors M Omega is far better conditioned than
// from a random block (Gram condition ~1e12-1e14 against ~1e17 on the vsa2m,
// vsa524k and ks200k inner matrices), within CholeskyQR's reach; the noise keeps
// every eigenvector's component in the start block nonzero.
__global__ void k_fill_start(double* __restrict__ Q, int r, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    uint64_t z = (uint64_t)e + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    Q[e] = (e % r == e / r ? 1.0 : 0.0) + 1e-3 * u;
}

// Fill the lower triangle of a column-major symmetric n x n matrix from its upper one.
__global__ void k_mirror_upper(double* __restrict__ A, int n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);
    if (i > j) A[e] = A[(int64_t)i * n + j];
}

// res[j] = |Z(:,j) - lam_j V(:,j)| / |lam_j| (infinite for lam_j = 0 or a NaN); one
// block per column.
__global__ void k_ritz_res(const double* __restrict__ Z, const double* __restrict__ V,
                           const double* __restrict__ lam, int r, double* __restrict__ res) {
    __shared__ double red[32];
    const int j = blockIdx.x;
    const double l = lam[j];
    double acc = 0.0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
        const double t = Z[(int64_t)j * r + i] - l * V[(int64_t)j * r + i];
        acc += t * t;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += red[q];
        const double q = sqrt(sum) / fabs(l);
        res[j] = q == q && l != 0.0 ? q : INFINITY;
    }
}

// Scale every column of the r x b matrix Y to unit 2-norm (one block per column;
// a zero column stays zero).
__global__ void k_unit_cols(double* __restrict__ Y, int r) {
    __shared__ double red[32];
    __shared__ double inv;
    double* y = Y + (int64_t)blockIdx.x * r;
    double acc = 0.0;
    for (int i = threadIdx.x; i < r; i += blockDim.x) acc += y[i] * y[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        inv = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) y[i] *= inv;
}

// ---------------------------------------------------------------------------
// FP64-accurate products of the r x r stage on the tensor cores (k_ozmm from
// seven-digit planes, ozmm.cu).  Operands are cut into K-major planes (K padded
// to 16) in the lift's plane buffer, idle until the lift; their row exponents go
// to rre.
// ---------------------------------------------------------------------------

// Planes of the rows of the column-major rows x cols matrix A (ld lda); K = cols.
static cudaError_t rr_row_planes(const double* A, int64_t lda, int rows, int cols, uint16_t* P, int* ex,
                                 double* rmax, cudaStream_t s) {
    const int ldk = lift_ldk(cols);
    k_rowmax_any<double><<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(A, lda, rows, cols, rmax);
    k_lift_planes<double, kDigits><<<dim3((unsigned)((ldk + 63) / 64), (unsigned)((rows + 31) / 32)), 256, 0, s>>>(
        A, lda, rows, cols, ldk, 0, rows, rows, rmax, reinterpret_cast<uint32_t*>(P), ex);
    return cudaGetLastError();
}

// Planes of the columns of the column-major rows x cols matrix A (ld rows): plane
// row j holds column j; K = rows.
static cudaError_t rr_col_planes(const double* A, int rows, int cols, uint16_t* P, int* ex, cudaStream_t s) {
    k_lift_ypl<kDigits><<<cols, 256, 0, s>>>(A, rows, cols, lift_ldk(rows), reinterpret_cast<uint32_t*>(P), ex);
    return cudaGetLastError();
}

// C(i, j) = sum_{c < K} A(i, c) B(j, c), i < m, j < n, into column-major C (ld
// ldc), from the planes of A's m rows and B's n rows.
static cudaError_t rr_product(const uint16_t* Pa, const int* ea, int m, const uint16_t* Pb, const int* eb, int n,
                              int K, double* C, int64_t ldc, int* flag, cudaStream_t s) {
    const int ldk = lift_ldk(K);
    CUtensorMap ma, mb;
    if (!ozmm_map(&ma, Pa, m, ldk, (int64_t)m * ldk, true) || !ozmm_map(&mb, Pb, n, ldk, (int64_t)n * ldk, false))
        return cudaErrorInvalidValue;
    return launch_ozmm(ma, mb, ea, 0, eb, 0, m, n, ldk, nullptr, C, ldc, 0, nullptr, 0, 0, flag, s);
}

// M = (R C) R^T (Section 2.2's inner matrix; R upper triangular with A = R^T R,
// strict lower triangle zero), both triangles.  R's row planes are the first
// product's A operand and the second's B operand.
static cudaError_t form_inner(const double* R, const double* C, int r, const EigWs& w, cudaStream_t s) {
    uint16_t* PR = w.lp;
    uint16_t* P1 = w.lp + (size_t)kDigits * r * lift_ldk(r);
    int* eR = w.rre;
    int* e1 = w.rre + r;
    cudaError_t e;
    if ((e = rr_row_planes(R, r, r, r, PR, eR, w.frow, s)) != cudaSuccess) return e;
    if ((e = rr_col_planes(C, r, r, P1, e1, s)) != cudaSuccess) return e;
    if ((e = rr_product(PR, eR, r, P1, e1, r, r, w.CZ, r, w.ozflag, s)) != cudaSuccess) return e;   // R C
    if ((e = rr_row_planes(w.CZ, r, r, r, P1, e1, w.frow, s)) != cudaSuccess) return e;
    return rr_product(P1, e1, r, PR, eR, r, r, w.M, r, w.ozflag, s);                                 // (R C) R^T
}

// CholeskyQR of Y (r x b), first half: columns scaled to unit norm (power steps
// leave Y's column norms spanning the spectrum of M; the Gram's condition then
// depends on the angles between columns only), G = Y^T Y on the tensor cores
// (planes of Y's columns in Py), G = R^T R (cuSOLVER potrf; *info > 0 if the
// Gram is numerically singular).
static int cholqr_factor(cusolverDnHandle_t h, double* Y, int r, int b, double* G, uint16_t* Py, int* ye,
                         double* work, int lwork, int* info, int* flag, cudaStream_t s) {
    k_unit_cols<<<b, 256, 0, s>>>(Y, r);
    KEVD_CUDA_TRY(rr_col_planes(Y, r, b, Py, ye, s));
    KEVD_CUDA_TRY(rr_product(Py, ye, b, Py, ye, b, r, G, b, flag, s));
    return cusolverDnDpotrf(h, CUBLAS_FILL_MODE_UPPER, b, G, b, work, lwork, info) == CUSOLVER_STATUS_SUCCESS
               ? KEVD_OK
               : KEVD_ECUDA;
}

// Second half: Y <- Y R^-1, an orthonormal basis of Y's columns (cuBLAS trsm).
static int cholqr_apply(cublasHandle_t hb, double* Y, int r, int b, const double* G) {
    const double one = 1.0;
    return cublasDtrsm(hb, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, r, b, &one, G,
                       b, Y, r) == CUBLAS_STATUS_SUCCESS
               ? KEVD_OK
               : KEVD_ECUDA;
}

// Householder QR of Y (r x b) in place: Y <- Q (cuSOLVER geqrf + orgqr), for a
// block whose Gram is too ill-conditioned for CholeskyQR.
static int householder_q(cusolverDnHandle_t h, double* Y, int r, int b, double* tau, double* work, int lwork,
                         int* info) {
    if (cusolverDnDgeqrf(h, r, b, Y, r, tau, work, lwork, info) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDorgqr(h, r, b, b, Y, r, tau, work, lwork, info) != CUSOLVER_STATUS_SUCCESS)
        return KEVD_ECUDA;
    return KEVD_OK;
}

// C (m x n) = op(A) B with cuBLAS (column-major, no transpose of B).
static int bgemm(cublasHandle_t hb, bool ta, int m, int n, int kk, const double* A, int lda, const double* B, int ldb,
                 double* C, int ldc) {
    const double one = 1.0, zero = 0.0;
    return cublasDgemm(hb, ta ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, m, n, kk, &one, A, lda, B, ldb, &zero, C, ldc) ==
                   CUBLAS_STATUS_SUCCESS
               ? KEVD_OK
               : KEVD_ECUDA;
}

// Power steps after Q = orth(M Omega) before the first Rayleigh-Ritz.  The
// slowest wanted direction converges by lambda_{b+1} / lambda_k per step: 0.09 on
// the vsa2m inner matrix (r = 1,848, k = 256, b = 544), where six steps leave
// |M v - theta v| / theta at ~4e-8.
constexpr int kSubspaceSteps = 6;
// A failed check continues the iteration on the same subspace for the steps that
// the observed rate rho = theta_b / theta_k says are missing, with a margin of 10,
// within these bounds; beyond them the caller's subset eigensolver is cheaper.
constexpr int kSubspaceMaxSteps = 30;
constexpr int kSubspaceMaxRR = 3;
constexpr double kRitzTol = 1e-6;

// M: full symmetric r x r.  Q, Y: r x b scratch.  Output lam (k, ascending) and
// V (r x k, same order) when *ok is set on return.  Planes: M's rows (r), Q's and
// Y's columns (b each) at w.lp, which holds 7 ldk (r + 2b) <= 14 r ldk elements.
static int subspace_topk(cusolverDnHandle_t h, cublasHandle_t hb, const double* M, int r, int k, int b, double* Q,
                         double* Y, double* V, double* lam, double* ss, double* work, int lwork, int* info,
                         const EigWs& w, cudaStream_t s, bool* ok) {
    *ok = false;
    double* G = ss;
    double* B = G + (size_t)b * b;
    double* theta = B + (size_t)b * b;
    double* Z = theta + b;
    double* res = Z + (size_t)r * k;
    double* tau = res + k;
    const size_t pl = (size_t)kDigits * lift_ldk(r);
    uint16_t* Pm = w.lp;
    uint16_t* Pq = Pm + pl * r;
    uint16_t* Py = Pq + pl * b;
    int* me = w.rre;
    int* qe = me + r;
    int* ye = qe + b;
    if (cublasSetStream(hb, s) != CUBLAS_STATUS_SUCCESS) return KEVD_ECUDA;
    const int64_t rb = (int64_t)r * b;
    k_fill_start<<<(unsigned)((rb + 255) / 256), 256, 0, s>>>(Q, r, rb);
    KEVD_CUDA_TRY(rr_col_planes(M, r, r, Pm, me, s));   // M symmetric: its columns are its rows
    auto mq = [&](const double* Qi, double* Yo) -> cudaError_t {   // Yo = M Qi; Qi's planes stay in Pq
        const cudaError_t e = rr_col_planes(Qi, r, b, Pq, qe, s);
        return e != cudaSuccess ? e : rr_product(Pm, me, r, Pq, qe, b, r, Yo, r, w.ozflag, s);
    };
    KEVD_CUDA_TRY(mq(Q, Y));   // Y = M Omega
    std::vector<double> hres(k), htheta(b);
    int orths = 0, target = kSubspaceSteps + 1;   // orthonormalisations: orth(M Omega) + power steps
    for (int rr_round = 0;; ++rr_round) {
        while (orths < target) {   // Y = M Q on entry: Q <- orth(Y), then the next product
            int st = cholqr_factor(h, Y, r, b, G, Py, ye, work, lwork, info, w.ozflag, s);
            if (st != KEVD_OK) return st;
            int pinfo = 0;
            if (orths == 0) {   // M Omega: columns spanning the whole spectrum of M may defeat CholeskyQR
                KEVD_CUDA_TRY(cudaMemcpyAsync(&pinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
                KEVD_CUDA_TRY(cudaStreamSynchronize(s));
            }
            if (pinfo != 0) {
                KEVD_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), s));
                st = householder_q(h, Y, r, b, tau, work, lwork, info);
            } else {
                st = cholqr_apply(hb, Y, r, b, G);
            }
            if (st != KEVD_OK) return st;
            std::swap(Q, Y);
            KEVD_CUDA_TRY(mq(Q, Y));
            ++orths;
        }
        KEVD_CUDA_TRY(rr_col_planes(Y, r, b, Py, ye, s));
        KEVD_CUDA_TRY(rr_product(Pq, qe, b, Py, ye, b, r, B, b, w.ozflag, s));   // B = Q^T M Q
        if (cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, b, B, b, theta, work, lwork, info) !=
            CUSOLVER_STATUS_SUCCESS)
            return KEVD_ECUDA;
        const double* Wk = B + (size_t)(b - k) * b;                          // top k Ritz vectors (ascending)
        int st = bgemm(hb, false, r, k, b, Q, r, Wk, b, V, r);               // V = Q W_k
        if (st == KEVD_OK) st = bgemm(hb, false, r, k, b, Y, r, Wk, b, Z, r);   // Z = M V
        if (st != KEVD_OK) return st;
        k_ritz_res<<<k, 256, 0, s>>>(Z, V, theta + (b - k), r, res);
        KEVD_CUDA_TRY(cudaGetLastError());
        int hinfo = 0, hoz = 0;
        KEVD_CUDA_TRY(cudaMemcpyAsync(hres.data(), res, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
        KEVD_CUDA_TRY(cudaMemcpyAsync(htheta.data(), theta, (size_t)b * sizeof(double), cudaMemcpyDeviceToHost, s));
        KEVD_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
        KEVD_CUDA_TRY(cudaMemcpyAsync(&hoz, w.ozflag, sizeof(int), cudaMemcpyDeviceToHost, s));
        KEVD_CUDA_TRY(cudaStreamSynchronize(s));
        if (hoz) return KEVD_ETIMEOUT;
        if (hinfo != 0) return KEVD_OK;   // not ok: the caller falls back
        double worst = 0.0;
        for (int j = 0; j < k; ++j) worst = std::max(worst, hres[j]);   // an infinite or NaN ratio stays
        if (worst <= kRitzTol) {
            KEVD_CUDA_TRY(cudaMemcpyAsync(lam, theta + (b - k), (size_t)k * sizeof(double), cudaMemcpyDeviceToDevice,
                                          s));
            *ok = true;
            return KEVD_OK;
        }
        const double rho = htheta[0] / htheta[b - k];
        if (rr_round + 1 >= kSubspaceMaxRR || !(worst < INFINITY) || !(rho > 0.0 && rho < 1.0)) return KEVD_OK;
        const double more = std::ceil(std::log(worst / (0.1 * kRitzTol)) / -std::log(rho));
        if (!(more >= 1.0) || orths + more > kSubspaceMaxSteps + 1) return KEVD_OK;
        target = orths + (int)more;
    }
}

// Cutoff of the Gram spectrum; Z = W diag(sqrt S) on kept directions.
__global__ void k_cutoff(const double* __restrict__ S, int r, double tau, double* sh, double* sih, int* kept) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const double smax = S[r - 1];
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const bool keep = smax > 0.0 && S[j] > tau * smax;
        sh[j] = keep ? sqrt(S[j]) : 0.0;
        sih[j] = keep ? 1.0 / sqrt(S[j]) : 0.0;
        if (keep) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *kept = cnt;
}

__global__ void k_scale_cols(const double* __restrict__ W, const double* __restrict__ sc, int r,
                             double* __restrict__ Z) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)r * r) Z[e] = W[e] * sc[e / r];
}

// Vt(:, j) = diag(sih) V(:, r-1-j), evals[j] = lam[r-1-j]  (descending order).
__global__ void k_select_top(const double* __restrict__ V, const double* __restrict__ lam,
                             const double* __restrict__ sih, int r, int k, double* __restrict__ Vt,
                             double* __restrict__ evals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)r * k) {
        const int c = (int)(e % r), j = (int)(e / r);
        Vt[e] = sih[c] * V[(int64_t)(r - 1 - j) * r + c];
    }
    if (e < k) evals[e] = lam[r - 1 - e];
}

// Zero the strictly lower triangle of a column-major r x r matrix.
__global__ void k_zero_lower(double* __restrict__ R, int r) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)r * r && (e % r) > (e / r)) R[e] = 0.0;
}

// Vt(:, j) = V(:, k-1-j), evals[j] = lam[k-1-j] for the k eigenpairs returned
// in ascending order by the subset eigensolver.
__global__ void k_select_subset(const double* __restrict__ V, const double* __restrict__ lam, int r, int k,
                                double* __restrict__ Vt, double* __restrict__ evals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)r * k) {
        const int c = (int)(e % r), j = (int)(e / r);
        Vt[e] = V[(int64_t)(k - 1 - j) * r + c];
    }
    if (e < k) evals[e] = lam[k - 1 - e];
}

// Vt(:, j) = V(:, k-1-j) / sqrt(lam[k-1-j]) (0 for non-positive), evals[j] = lam[k-1-j].
__global__ void k_select_sym(const double* __restrict__ V, const double* __restrict__ lam, int r, int k,
                             double* __restrict__ Vt, double* __restrict__ evals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)r * k) {
        const int c = (int)(e % r), j = (int)(e / r);
        const double l = lam[k - 1 - j];
        Vt[e] = l > 0.0 ? V[(int64_t)(k - 1 - j) * r + c] / sqrt(l) : 0.0;
    }
    if (e < k) evals[e] = lam[k - 1 - e];
}

__global__ void k_sqrt(const double* __restrict__ x, int64_t N, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] = sqrt(x[i]);
}

__global__ void k_set_const_col(double* __restrict__ U, int64_t N, double v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) U[i] = v;
}

// Per column: entry of largest magnitude, lowest index on ties (cmax = its signed
// value, cidx = its index); k_colsign then flips the column so that entry is
// positive.  Magnitudes compare as the integer bits of |x| (monotone for
// non-negative doubles; no FP64 compare on the slow pipe).  A 16-byte aligned
// column is read as four 16-byte vectors per thread per step (eight loads in
// flight), the rest element by element.
__device__ __forceinline__ void key_merge(unsigned long long& k, int64_t& i, unsigned long long k2, int64_t i2) {
    if (k2 > k || (k2 == k && i2 < i)) {
        k = k2;
        i = i2;
    }
}

__global__ void __launch_bounds__(1024) k_colmax(const double* __restrict__ U, int64_t N, double* cmax,
                                                 int64_t* cidx) {
    __shared__ unsigned long long sk[32];
    __shared__ int64_t si[32];
    const int j = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double* col = U + (int64_t)j * N;
    constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long key = 0;
    int64_t idx = LLONG_MAX;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(col) & 15) == 0) {
        const double2* c2 = reinterpret_cast<const double2*>(col);
        const int64_t n2 = N / 2, T = blockDim.x;
        int64_t p = threadIdx.x;
        for (; p + 3 * T < n2; p += 4 * T) {
            double2 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = c2[p + u * T];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = 2 * (p + u * T);
                key_merge(key, idx, (unsigned long long)__double_as_longlong(x[u].x) & kAbs, e);
                key_merge(key, idx, (unsigned long long)__double_as_longlong(x[u].y) & kAbs, e + 1);
            }
        }
        for (; p < n2; p += T) {
            const double2 x = c2[p];
            key_merge(key, idx, (unsigned long long)__double_as_longlong(x.x) & kAbs, 2 * p);
            key_merge(key, idx, (unsigned long long)__double_as_longlong(x.y) & kAbs, 2 * p + 1);
        }
        done = 2 * n2;
    }
    for (int64_t i = done + threadIdx.x; i < N; i += blockDim.x)
        key_merge(key, idx, (unsigned long long)__double_as_longlong(col[i]) & kAbs, i);
#pragma unroll
    for (int o = 16; o; o >>= 1)
        key_merge(key, idx, __shfl_xor_sync(0xffffffffu, key, o), __shfl_xor_sync(0xffffffffu, idx, o));
    if (lane == 0) {
        sk[wid] = key;
        si[wid] = idx;
    }
    __syncthreads();
    if (wid == 0) {
        key = lane < (int)(blockDim.x >> 5) ? sk[lane] : 0;
        idx = lane < (int)(blockDim.x >> 5) ? si[lane] : LLONG_MAX;
#pragma unroll
        for (int o = 16; o; o >>= 1)
            key_merge(key, idx, __shfl_xor_sync(0xffffffffu, key, o), __shfl_xor_sync(0xffffffffu, idx, o));
        if (lane == 0) {
            cmax[j] = col[idx];   // signed value of the pivot entry
            cidx[j] = idx;
        }
    }
}

__global__ void k_colsign(double* __restrict__ U, int64_t N, const double* __restrict__ cval) {
    const int j = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && cval[j] < 0.0) U[(int64_t)j * N + i] = -U[(int64_t)j * N + i];
}


// Lift U = D~^-1 F Y, sign convention, solver status; kept_fixed >= 0 reports
// that count instead of the spectral cutoff's.  With lm, F is the low-memory
// factor's K(:,S) W^-T, rebuilt panel by panel (lowmem.cu).
static int lift_and_finish(const void* F, int f_dtype, int64_t N, int r, int64_t ldf, const double* dtil, int k,
                           double* U, int32_t* kept, int kept_fixed, const EigWs& w, cudaStream_t s,
                           const KevdLowmemLift* lm) {
    if (lm) {
        const int st = kevd_lowmem_lift(*lm, N, r, k, w.Y, dtil, U, s);
        if (st != KEVD_OK) return st;
    } else {
        TraceScope tr(kStLift, s);
        if (f_dtype == KEVD_F32)
            KEVD_CUDA_TRY(lift_fp32(N, k, r, static_cast<const float*>(F), ldf, w.Y, U, dtil, w, s));   // U = D~^-1 F Y
        else
            KEVD_CUDA_TRY(lift_fp64(N, k, r, static_cast<const double*>(F), ldf, w.Y, U, dtil, w, s));   // U = D~^-1 F Y
    }
    {
        TraceScope tr(kStOther, s);
        k_colmax<<<k, 1024, 0, s>>>(U, N, w.cmax, w.cidx);
        k_colsign<<<dim3((unsigned)((N + 255) / 256), k), 256, 0, s>>>(U, N, w.cmax);
    }
    KEVD_LAUNCH_CHECK();
    int hinfo[4] = {0, 0, 0, 0}, hoz = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(hinfo, w.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaMemcpyAsync(&hoz, w.ozflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    if (kept) *kept = kept_fixed >= 0 ? kept_fixed : hinfo[2];
    if (hoz) return KEVD_ETIMEOUT;
    if (hinfo[0] != 0 || hinfo[1] != 0 || hinfo[3] != 0) return KEVD_EEIG;
    return KEVD_OK;
}

}  // namespace kevd

using namespace kevd;

size_t kevd_eig_ws(int64_t N, int32_t r, int32_t k) {
    if (r < 1 || k < 1 || k > r) return 0;
    const int64_t lwork = solver_lwork(r, k, nullptr);
    if (lwork < 0) return 0;
    size_t bytes = 0;
    carve_eig(nullptr, N, r, k, lwork, &bytes);
    return bytes;
}

// The r x r stage of eig_topk and eig_topk_lowmem (arguments checked by the
// callers); lm_in selects the low-memory lift, whose panel workspace follows
// the eigen workspace.
static int eig_topk_impl(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf, const double* dtil,
                         const double* A, const double* C, int32_t k, double tau, double* evals, double* U,
                         int32_t* kept, void* workspace, size_t ws_bytes, void* stream,
                         const KevdLowmemLift* lm_in) {
    cusolverDnHandle_t h = solver_handle();
    if (!h) return KEVD_ECUDA;
    const int64_t lwork = solver_lwork(rank, k, nullptr);
    if (lwork < 0) return KEVD_ECUDA;
    size_t need = 0;
    EigWs w = carve_eig(workspace, N, rank, k, lwork, &need);
    const size_t extra = lm_in ? kevd_lowmem_lift_bytes(N, lm_in->d, rank) : 0;
    if (!workspace || ws_bytes < need + extra || (reinterpret_cast<uintptr_t>(workspace) % kAlign))
        return KEVD_EWORKSPACE;
    KevdLowmemLift lm_local;
    const KevdLowmemLift* lm = nullptr;
    if (lm_in) {
        lm_local = *lm_in;
        lm_local.ws = static_cast<char*>(workspace) + need;
        lm = &lm_local;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cusolverDnSetStream(h, s) != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
    const int r = rank;
    const int64_t rr = (int64_t)r * r;

    cusolverStatus_t cs;
    KEVD_CUDA_TRY(cudaMemsetAsync(w.ozflag, 0, sizeof(int), s));
    // ---- Cholesky route ----
    KEVD_CUDA_TRY(cudaMemcpyAsync(w.W, A, rr * sizeof(double), cudaMemcpyDeviceToDevice, s));
    KEVD_CUDA_TRY(cudaMemsetAsync(w.info, 0, 4 * sizeof(int), s));
    {
        TraceScope tr(kStSolver, s);
        cs = cusolverDnDpotrf(h, CUBLAS_FILL_MODE_UPPER, r, w.W, r, w.work, (int)lwork, w.info);
    }
    if (cs != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
    int pinfo = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&pinfo, w.info, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    if (pinfo == 0) {
        {
            TraceScope tr(kStOther, s);
            k_zero_lower<<<(unsigned)((rr + 255) / 256), 256, 0, s>>>(w.W, r);
            KEVD_CUDA_TRY(form_inner(w.W, C, r, w, s));   // M = (R C) R^T
        }
        KEVD_LAUNCH_CHECK();
        const double* Vk = w.M;   // the k eigenvectors, ascending, first k columns
        bool done = false;
        const int sb = subspace_b(r, k);
        // KEVD_TOPK=full: the subset eigensolver (comparisons); KEVD_TOPK=subspace: the
        // precision form's subspace solver, whose failed check is then an error
        const char* topk_env = getenv("KEVD_TOPK");
        const bool full = topk_env && std::strcmp(topk_env, "full") == 0;
        const bool strict = topk_env && std::strcmp(topk_env, "subspace") == 0;
        if (strict && (f_dtype != KEVD_F32 || sb == 0 || use_native_syev(r))) return KEVD_EEIG;
        if (f_dtype == KEVD_F32 && sb > 0 && !full && !use_native_syev(r)) {
            cublasHandle_t hb = blas_handle();
            if (!hb) return KEVD_ECUDA;
            TraceScope tr(kStSolver, s);
            k_mirror_upper<<<(unsigned)((rr + 255) / 256), 256, 0, s>>>(w.M, r);
            const int st = subspace_topk(h, hb, w.M, r, k, sb, w.Z, w.CZ, w.Vt, w.lam, w.ss, w.work, (int)lwork,
                                         w.info + 1, w, s, &done);
            if (st != KEVD_OK) return st;
            if (done) Vk = w.Vt;
            else if (strict) return KEVD_EEIG;
        }
        if (done) {
        } else if (use_native_syev(r)) {
            cublasHandle_t hb = blas_handle();
            if (!hb) return KEVD_ECUDA;
            const int st = kevd_syev_topk(h, hb, w.M, r, k, w.lam, w.CZ, w.sy, w.work, (int)lwork, w.info + 1, s);
            if (st != KEVD_OK) return st;
            Vk = w.CZ;
        } else {
            int meig = 0;
            TraceScope tr(kStSolver, s);
            cs = cusolverDnDsyevdx(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER, r, w.M,
                                   r, 0.0, 0.0, r - k + 1, r, &meig, w.lam, w.work, (int)lwork, w.info + 1);
            if (cs != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
        }
        {
            TraceScope tr(kStOther, s);
            k_select_subset<<<(unsigned)(((int64_t)r * k + 255) / 256), 256, 0, s>>>(Vk, w.lam, r, k, w.Y, evals);
        }
        KEVD_LAUNCH_CHECK();
        {
            TraceScope tr(kStSolver, s);   // Y = R^-1 V_k by back substitution (in place)
            cublasHandle_t hb = blas_handle();
            const double one = 1.0;
            if (!hb || cublasSetStream(hb, s) != CUBLAS_STATUS_SUCCESS ||
                cublasDtrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, r, k, &one,
                            w.W, r, w.Y, r) != CUBLAS_STATUS_SUCCESS)
                return KEVD_ECUDA;
        }
        return lift_and_finish(F, f_dtype, N, r, ldf, dtil, k, U, kept, r, w, s, lm);
    }

    // ---- spectral route (A numerically singular) ----
    KEVD_CUDA_TRY(cudaMemcpyAsync(w.W, A, rr * sizeof(double), cudaMemcpyDeviceToDevice, s));
    KEVD_CUDA_TRY(cudaMemsetAsync(w.info, 0, 4 * sizeof(int), s));
    {
        TraceScope tr(kStSolver, s);
        cs = cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, r, w.W, r, w.S, w.work, (int)lwork,
                              w.info);
    }
    if (cs != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
    {
        TraceScope tr(kStOther, s);
        k_cutoff<<<1, 1024, 0, s>>>(w.S, r, tau, w.sh, w.sih, w.info + 2);
        k_scale_cols<<<(unsigned)((rr + 255) / 256), 256, 0, s>>>(w.W, w.sh, r, w.Z);
        dgemm(false, r, r, r, C, r, w.Z, r, w.CZ, r, nullptr, s);       // C Z
        dgemm(true, r, r, r, w.Z, r, w.CZ, r, w.M, r, nullptr, s);      // Z^T (C Z)
    }
    KEVD_LAUNCH_CHECK();
    {
        TraceScope tr(kStSolver, s);
        cs = cusolverDnDsyevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, r, w.M, r, w.lam, w.work,
                              (int)lwork, w.info + 1);
    }
    if (cs != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
    {
        TraceScope tr(kStOther, s);
        k_select_top<<<(unsigned)(((int64_t)r * k + 255) / 256), 256, 0, s>>>(w.M, w.lam, w.sih, r, k, w.Vt, evals);
        dgemm(false, r, k, r, w.W, r, w.Vt, r, w.Y, r, nullptr, s);     // Y = W diag(sih) V_k
    }
    KEVD_LAUNCH_CHECK();
    return lift_and_finish(F, f_dtype, N, r, ldf, dtil, k, U, kept, -1, w, s, lm);
}


extern "C" int eig_topk(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf, const double* dtil,
                        const double* A, const double* C, int32_t k, double tau, double* evals, double* U,
                        int32_t* kept, void* workspace, size_t ws_bytes, void* stream) {
    if (!F || !dtil || !A || !C || !evals || !U) return KEVD_EINVAL;
    if (N < 1 || rank < 1 || rank > N || ldf < N || k < 1 || k > rank) return KEVD_EINVAL;
    if (f_dtype != KEVD_F64 && f_dtype != KEVD_F32) return KEVD_EINVAL;
    if (!(tau >= 0.0 && tau < 1.0)) return KEVD_EINVAL;
    return eig_topk_impl(F, f_dtype, N, rank, ldf, dtil, A, C, k, tau, evals, U, kept, workspace, ws_bytes, stream,
                         nullptr);
}

size_t kevd_lowmem_eig_ws(int64_t N, int32_t d, int32_t r, int32_t k) {
    const size_t e = kevd_eig_ws(N, r, k);
    if (e == 0 || d < 1) return 0;
    return e + kevd_lowmem_lift_bytes(N, d, r);
}

extern "C" int eig_topk_lowmem(const double* X, int64_t N, int32_t d, double eps, const int64_t* pivots,
                               const double* W, int64_t ldw, int32_t rank, const double* dtil, const double* A,
                               const double* C, int32_t k, double tau, double* evals, double* U, int32_t* kept,
                               void* workspace, size_t ws_bytes, void* stream) {
    if (!X || !pivots || !W || !dtil || !A || !C || !evals || !U) return KEVD_EINVAL;
    if (N < 1 || N > INT_MAX || d < 1 || rank < 1 || rank > N || ldw < rank || ldw > INT_MAX || k < 1 || k > rank)
        return KEVD_EINVAL;
    if (!(eps > 0.0) || !isfinite(eps) || !(tau >= 0.0 && tau < 1.0)) return KEVD_EINVAL;
    KevdLowmemLift lm{X, d, 1.0 / eps, pivots, W, ldw, nullptr};
    return eig_topk_impl(nullptr, KEVD_F64, N, rank, N, dtil, A, C, k, tau, evals, U, kept, workspace, ws_bytes,
                         stream, &lm);
}

using namespace kevd;

// ---------------------------------------------------------------------------
// Symmetric normalisation (Section 2.1): top-k eigenpairs of
// L~ = B B^T, B = D~^-1/2 F, from A_s = B^T B = V Lambda V^T:
// U = B V Lambda^-1/2 = D~^-1/2 F (V Lambda^-1/2).
// ---------------------------------------------------------------------------
extern "C" int symmetric_eig_topk(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf,
                                  const double* dtil, const double* As, int32_t k, double* evals, double* U,
                                  void* workspace, size_t ws_bytes, void* stream) {
    if (!F || !dtil || !As || !evals || !U) return KEVD_EINVAL;
    if (N < 1 || rank < 1 || rank > N || ldf < N || k < 1 || k > rank) return KEVD_EINVAL;
    if (f_dtype != KEVD_F64 && f_dtype != KEVD_F32) return KEVD_EINVAL;
    cusolverDnHandle_t h = solver_handle();
    if (!h) return KEVD_ECUDA;
    const int64_t lwork = solver_lwork(rank, k, nullptr);
    if (lwork < 0) return KEVD_ECUDA;
    size_t need = 0;
    EigWs w = carve_eig(workspace, N, rank, k, lwork, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cusolverDnSetStream(h, s) != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
    const int r = rank;
    KEVD_CUDA_TRY(cudaMemcpyAsync(w.W, As, (size_t)r * r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    KEVD_CUDA_TRY(cudaMemsetAsync(w.ozflag, 0, sizeof(int), s));
    KEVD_CUDA_TRY(cudaMemsetAsync(w.info, 0, 4 * sizeof(int), s));
    const double* Vk = w.W;
    if (use_native_syev(r)) {
        cublasHandle_t hb = blas_handle();
        if (!hb) return KEVD_ECUDA;
        const int st = kevd_syev_topk(h, hb, w.W, r, k, w.lam, w.CZ, w.sy, w.work, (int)lwork, w.info + 1, s);
        if (st != KEVD_OK) return st;
        Vk = w.CZ;
    } else {
        int meig = 0;
        TraceScope tr(kStSolver, s);
        const cusolverStatus_t cs = cusolverDnDsyevdx(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                                      CUBLAS_FILL_MODE_UPPER, r, w.W, r, 0.0, 0.0, r - k + 1, r, &meig,
                                                      w.lam, w.work, (int)lwork, w.info + 1);
        if (cs != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
    }
    {
        TraceScope tr(kStOther, s);
        k_select_sym<<<(unsigned)(((int64_t)r * k + 255) / 256), 256, 0, s>>>(Vk, w.lam, r, k, w.Y, evals);
        k_sqrt<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(dtil, N, w.rowdiv);
    }
    KEVD_LAUNCH_CHECK();
    {
        TraceScope tr(kStLift, s);
        if (f_dtype == KEVD_F32)
            KEVD_CUDA_TRY(lift_fp32(N, k, r, static_cast<const float*>(F), ldf, w.Y, U, w.rowdiv, w, s));
        else
            KEVD_CUDA_TRY(lift_fp64(N, k, r, static_cast<const double*>(F), ldf, w.Y, U, w.rowdiv, w, s));
    }
    {
        TraceScope tr(kStOther, s);
        k_colmax<<<k, 1024, 0, s>>>(U, N, w.cmax, w.cidx);
        k_colsign<<<dim3((unsigned)((N + 255) / 256), k), 256, 0, s>>>(U, N, w.cmax);
    }
    KEVD_LAUNCH_CHECK();
    int hinfo[4] = {0, 0, 0, 0}, hoz = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(hinfo, w.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaMemcpyAsync(&hoz, w.ozflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    if (hoz) return KEVD_ETIMEOUT;
    return hinfo[1] != 0 ? KEVD_EEIG : KEVD_OK;
}

// ---------------------------------------------------------------------------
// Optional last step of Algorithm 1: U(:,0) = 1_N / sqrt(N), then
// re-orthonormalise the columns (CholeskyQR2: G = U^T U = R^T R, U <- U R^-1,
// twice; Q has the positive-diagonal R of the QR factorisation).
// ---------------------------------------------------------------------------
namespace {
struct FixWs {
    double* G;      // k x k
    double* T;      // N x k
    double* gpart;
    double* work;
    int* info;
};
FixWs carve_fix(void* base, int64_t N, int k, int64_t lwork, size_t* bytes) {
    Carver c(base);
    FixWs w;
    w.G = c.take<double>((size_t)k * k);
    w.T = c.take<double>((size_t)N * k);
    w.gpart = c.take<double>(kevd_gram_partial_doubles(N, k));
    w.work = c.take<double>((size_t)std::max<int64_t>(lwork, 1));
    w.info = c.take<int>(4);
    *bytes = c.off;
    return w;
}
int64_t fix_lwork(int k, size_t* th) {
    cusolverDnHandle_t h = solver_handle();
    if (!h) return -1;
    int l = 0;
    if (cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_UPPER, k, nullptr, k, &l) != CUSOLVER_STATUS_SUCCESS) return -1;
    size_t td = 0;
    if (cusolverDnXtrtri_bufferSize(h, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, k, CUDA_R_64F, nullptr, k, &td,
                                    th) != CUSOLVER_STATUS_SUCCESS)
        return -1;
    return std::max<int64_t>(l, (int64_t)((td + 7) / 8));
}
}  // namespace

size_t kevd_fix_ws(int64_t N, int32_t k) {
    if (N < 1 || k < 1 || k > N) return 0;
    size_t th = 0;
    const int64_t lw = fix_lwork(k, &th);
    if (lw < 0) return 0;
    size_t bytes = 0;
    carve_fix(nullptr, N, k, lw, &bytes);
    return bytes;
}

extern "C" int constant_eigvec_fix(double* U, int64_t N, int32_t k, void* workspace, size_t ws_bytes, void* stream) {
    if (!U || N < 1 || k < 1 || k > N) return KEVD_EINVAL;
    cusolverDnHandle_t h = solver_handle();
    if (!h) return KEVD_ECUDA;
    size_t th = 0;
    const int64_t lw = fix_lwork(k, &th);
    if (lw < 0) return KEVD_ECUDA;
    size_t need = 0;
    FixWs w = carve_fix(workspace, N, k, lw, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cusolverDnSetStream(h, s) != CUSOLVER_STATUS_SUCCESS) return KEVD_ECUDA;
    std::vector<char> hbuf(th + 16);
    KEVD_CUDA_TRY(cudaMemsetAsync(w.info, 0, 4 * sizeof(int), s));
    k_set_const_col<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(U, N, 1.0 / sqrt((double)N));
    for (int pass = 0; pass < 2; ++pass) {
        KEVD_CUDA_TRY(kevd_gram_plain(U, N, N, k, w.G, w.gpart, s));
        if (cusolverDnDpotrf(h, CUBLAS_FILL_MODE_UPPER, k, w.G, k, w.work, (int)lw, w.info + pass) !=
            CUSOLVER_STATUS_SUCCESS)
            return KEVD_ECUDA;
        k_zero_lower<<<(unsigned)(((int64_t)k * k + 255) / 256), 256, 0, s>>>(w.G, k);
        if (cusolverDnXtrtri(h, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, k, CUDA_R_64F, w.G, k, w.work,
                             (size_t)lw * sizeof(double), hbuf.data(), th, w.info + 2) != CUSOLVER_STATUS_SUCCESS)
            return KEVD_ECUDA;
        dgemm(false, N, k, k, U, N, w.G, k, w.T, N, nullptr, s);   // U R^-1
        KEVD_CUDA_TRY(cudaMemcpyAsync(U, w.T, (size_t)N * k * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    KEVD_LAUNCH_CHECK();
    int hinfo[4] = {0, 0, 0, 0};
    KEVD_CUDA_TRY(cudaMemcpyAsync(hinfo, w.info, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    return (hinfo[0] || hinfo[1] || hinfo[2]) ? KEVD_EEIG : KEVD_OK;
}
