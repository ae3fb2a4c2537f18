// bistoch_normalize: degree vectors and weighted Gram matrices of the
// bistochastic normalisation (Section 2.2; Algorithm 1), FP64 path.
//
//   s  = F^T 1          column sums, split over row ranges, fixed-order reduce
//   d~ = F s            row-local dot products (coalesced over rows)
//   t  = F^T d~^-1      as s, rows weighted by 1/d~
//   q~ = F t
//   A  = F^T diag(d~^-2) F,  C = F^T diag(q~^-1) F   in one pass: upper-triangle
//        64 x 64 output tiles x row splits, both Grams from the same staged
//        panels, fixed-order split reduction, mirrored to exact symmetry.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "trace.cuh"

namespace kevd {

constexpr int kGT = 64;   // Gram output tile
constexpr int kGK = 16;   // rows per staged chunk

struct NormWs {
    double* part;   // ncs x rank column-sum partials
    double* svec;   // rank
    double* tvec;   // rank
    int* flags;     // bit 0: some d~ <= 0, bit 1: some q~ <= 0
    double* wa;     // N: 1 / d~_i^2
    double* wc;     // N: 1 / q~_i
    float* waf;     // N: FP32 copies of the Gram weights (FP32 path)
    float* wcf;
    double* gpart;  // nsplit x ntri x 2 x 64 x 64 Gram partials
};

static int colsum_splits(int64_t N) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 4096)); }

static int gram_splits(int64_t N, int64_t ntri) {
    int64_t s = (1216 + ntri - 1) / ntri;
    s = std::min<int64_t>(s, std::max<int64_t>(1, N / 512));
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, 64));
}

static NormWs carve_norm(void* base, int64_t N, int rank, size_t* bytes) {
    Carver c(base);
    const int64_t nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
    NormWs w;
    w.part = c.take<double>((size_t)colsum_splits(N) * rank);
    w.svec = c.take<double>(rank);
    w.tvec = c.take<double>(rank);
    w.flags = c.take<int>(4);
    w.wa = c.take<double>(N);
    w.wc = c.take<double>(N);
    w.waf = c.take<float>(N);
    w.wcf = c.take<float>(N);
    w.gpart = c.take<double>((size_t)gram_splits(N, ntri) * ntri * 2 * kGT * kGT);
    *bytes = c.off;
    return w;
}

// Partial column sums of F, rows weighted by wmul_i when wmul != nullptr.
// Block: 8 warps = 8 columns; blockIdx.y = row split of `per` rows (a multiple
// of 32 * V * 4).  With V > 1 each lane loads V consecutive rows as one
// 16-byte vector.  FP32 factors are summed in FP32 over blocks of 4 vectors
// per lane and the block sums are added in FP64; FP64 factors in FP64.
template <typename T, int V>
__global__ void __launch_bounds__(256) k_colsum_partial(const T* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                                        int64_t per, const double* __restrict__ wmul,
                                                        double* __restrict__ part) {
    using VT = typename std::conditional<V == 1, T,
               typename std::conditional<std::is_same<T, float>::value, float4, double2>::type>::type;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= rank) return;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const T* col = F + (int64_t)c * ldf;
    double acc = 0.0;
    constexpr int STEP = 32 * V;
    int64_t i = i0 + lane * V;
    for (; i + 3 * STEP + V <= i1; i += 4 * STEP) {
        VT x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = *reinterpret_cast<const VT*>(col + i + u * STEP);
        T blk = T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T* e = reinterpret_cast<const T*>(&x[u]);
#pragma unroll
            for (int q = 0; q < V; ++q) blk += wmul ? e[q] * (T)wmul[i + u * STEP + q] : e[q];
        }
        acc += (double)blk;
    }
    for (; i < i1; i += STEP)
        for (int q = 0; q < V && i + q < i1; ++q) acc += wmul ? (double)col[i + q] * wmul[i + q] : (double)col[i + q];
    acc = warp_sum(acc);
    if (lane == 0) part[(size_t)blockIdx.y * rank + c] = acc;
}

__global__ void k_colsum_final(const double* __restrict__ part, int nsplit, int rank, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= rank) return;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += part[(size_t)q * rank + c];
    out[c] = s;
}

__global__ void k_recip(const double* __restrict__ x, int64_t N, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] = 1.0 / x[i];
}

__global__ void k_recip_f(const double* __restrict__ x, int64_t N, float* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] = (float)(1.0 / x[i]);
}

// out_i = F(i,:) . v ; flag bit if out_i <= 0 (or not a number).  Each thread
// owns V consecutive rows (one 16-byte vector per column when V > 1).  FP32
// factors: FP32 products summed over blocks of 32 columns, block sums in FP64.
template <typename T, int V>
__global__ void __launch_bounds__(256) k_rowdot(const T* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                                const double* __restrict__ v, double* __restrict__ out, int* flags,
                                                int bit) {
    using VT = typename std::conditional<V == 1, T,
               typename std::conditional<std::is_same<T, float>::value, float4, double2>::type>::type;
    extern __shared__ double vs_raw[];
    T* vs = reinterpret_cast<T*>(vs_raw);
    for (int c = threadIdx.x; c < rank; c += blockDim.x) vs[c] = (T)v[c];
    __syncthreads();
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V;
    if (i >= N) return;
    double acc[V];
#pragma unroll
    for (int q = 0; q < V; ++q) acc[q] = 0.0;
    if (i + V <= N) {
        for (int c0 = 0; c0 < rank; c0 += 32) {
            const int c1 = min(c0 + 32, rank);
            T blk[V];
#pragma unroll
            for (int q = 0; q < V; ++q) blk[q] = T(0);
            int c = c0;
            for (; c + 4 <= c1; c += 4) {
                VT x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = *reinterpret_cast<const VT*>(F + (int64_t)(c + u) * ldf + i);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const T* e = reinterpret_cast<const T*>(&x[u]);
#pragma unroll
                    for (int q = 0; q < V; ++q) blk[q] = fma(e[q], vs[c + u], blk[q]);
                }
            }
            for (; c < c1; ++c) {
                const VT x = *reinterpret_cast<const VT*>(F + (int64_t)c * ldf + i);
                const T* e = reinterpret_cast<const T*>(&x);
#pragma unroll
                for (int q = 0; q < V; ++q) blk[q] = fma(e[q], vs[c], blk[q]);
            }
#pragma unroll
            for (int q = 0; q < V; ++q) acc[q] += (double)blk[q];
        }
    } else {
        for (int c = 0; c < rank; ++c)
            for (int q = 0; q < V && i + q < N; ++q) acc[q] = fma((double)F[(int64_t)c * ldf + i + q], v[c], acc[q]);
    }
    for (int q = 0; q < V && i + q < N; ++q) {
        out[i + q] = acc[q];
        if (!(acc[q] > 0.0)) atomicOr(flags, bit);
    }
}

// Row weights of the two Grams: 1/d~^2 and 1/q~ (one division each per row).
__global__ void k_gram_weights(const double* __restrict__ dtil, const double* __restrict__ qtil, int64_t N,
                               double* __restrict__ wa, double* __restrict__ wc, float* __restrict__ waf,
                               float* __restrict__ wcf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double d = dtil[i];
    wa[i] = 1.0 / (d * d);
    wc[i] = 1.0 / qtil[i];
    waf[i] = (float)wa[i];
    wcf[i] = (float)wc[i];
}

// Upper-triangular tile index -> (I, J), I <= J.
__device__ __forceinline__ void tri_decode(int t, int nb, int& I, int& J) {
    I = 0;
    int rowlen = nb;
    while (t >= rowlen) {
        t -= rowlen;
        ++I;
        --rowlen;
    }
    J = I + t;
}

// Weighted Gram partials.  Block = one (I, J) tile and one row split; 256
// threads, 4 x 4 outputs per thread for each of A and C.
// T: element type of F; A: arithmetic of the products (double for FP64 F,
// float for FP32 F: FFMA with FP32 accumulation over one row split, FP64 across
// splits in k_gram_final).
// With wc == nullptr only the first Gram is formed (the second partial is zero).
template <typename T, typename A>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                              const A* __restrict__ wa, const A* __restrict__ wc,
                                              double* __restrict__ gpart, int nb, int ntri) {
    const bool two = wc != nullptr;
    using A2 = typename std::conditional<std::is_same<A, double>::value, double2, float2>::type;
    constexpr int P = kGT + 4;
    __shared__ __align__(16) A Ua[kGK][P];   // F(:,I) * wa
    __shared__ __align__(16) A Uc[kGK][P];   // F(:,I) * wc
    __shared__ __align__(16) A V[kGK][P];    // F(:,J)
    int I, J;
    tri_decode(blockIdx.x, nb, I, J);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t per = (N + gridDim.y - 1) / gridDim.y;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    A aa[4][4], ac[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) aa[a][c] = ac[a][c] = A(0);

    for (int64_t r0 = i0; r0 < i1; r0 += kGK) {
#pragma unroll
        for (int p = 0; p < (kGK * kGT) / 256; ++p) {
            const int e = tid + 256 * p, kk = e % kGK, col = e / kGK;
            const int64_t row = r0 + kk;
            const int ci = I * kGT + col, cj = J * kGT + col;
            A fi = A(0), fj = A(0), a = A(0), c = A(0);
            if (row < i1) {
                if (ci < rank) fi = (A)F[(int64_t)ci * ldf + row];
                if (cj < rank) fj = (A)F[(int64_t)cj * ldf + row];
                a = wa ? wa[row] : A(1);
                c = two ? wc[row] : A(0);
            }
            Ua[kk][col] = fi * a;
            Uc[kk][col] = fi * c;
            V[kk][col] = fj;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            const A2 ua0 = *reinterpret_cast<const A2*>(&Ua[kk][ty * 4]);
            const A2 ua1 = *reinterpret_cast<const A2*>(&Ua[kk][ty * 4 + 2]);
            const A2 uc0 = *reinterpret_cast<const A2*>(&Uc[kk][ty * 4]);
            const A2 uc1 = *reinterpret_cast<const A2*>(&Uc[kk][ty * 4 + 2]);
            const A2 v0 = *reinterpret_cast<const A2*>(&V[kk][tx * 4]);
            const A2 v1 = *reinterpret_cast<const A2*>(&V[kk][tx * 4 + 2]);
            const A a4[4] = {ua0.x, ua0.y, ua1.x, ua1.y};
            const A c4[4] = {uc0.x, uc0.y, uc1.x, uc1.y};
            const A v4[4] = {v0.x, v0.y, v1.x, v1.y};
            if (two) {
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        aa[a][c] = fma(a4[a], v4[c], aa[a][c]);
                        ac[a][c] = fma(c4[a], v4[c], ac[a][c]);
                    }
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) aa[a][c] = fma(a4[a], v4[c], aa[a][c]);
            }
        }
        __syncthreads();
    }
    double* out = gpart + ((size_t)blockIdx.y * ntri + blockIdx.x) * 2 * kGT * kGT;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            out[(ty * 4 + a) * kGT + tx * 4 + c] = (double)aa[a][c];
            out[kGT * kGT + (ty * 4 + a) * kGT + tx * 4 + c] = (double)ac[a][c];
        }
}

// Sum the split partials in order; write (I-row a, J-col c) and its mirror.
// Diagonal tiles keep their upper triangle only, so A and C are exactly symmetric.
__global__ void k_gram_final(const double* __restrict__ gpart, int nsplit, int ntri, int nb, int rank,
                             double* __restrict__ A, double* __restrict__ C) {
    const int t = blockIdx.x;
    int I, J;
    tri_decode(t, nb, I, J);
    for (int e = threadIdx.x; e < kGT * kGT; e += blockDim.x) {
        const int a = e / kGT, c = e % kGT;
        const int ra = I * kGT + a, rc = J * kGT + c;
        if (ra >= rank || rc >= rank) continue;
        if (I == J && a > c) continue;
        double sa = 0.0, sc = 0.0;
        for (int q = 0; q < nsplit; ++q) {
            const double* p = gpart + ((size_t)q * ntri + t) * 2 * kGT * kGT;
            sa += p[e];
            sc += p[kGT * kGT + e];
        }
        A[(int64_t)rc * rank + ra] = sa;
        A[(int64_t)ra * rank + rc] = sa;
        if (C) {
            C[(int64_t)rc * rank + ra] = sc;
            C[(int64_t)ra * rank + rc] = sc;
        }
    }
}

}  // namespace kevd

using namespace kevd;

size_t kevd_normalize_ws(int64_t N, int32_t rank) {
    if (N < 1 || rank < 1) return 0;
    size_t bytes = 0;
    carve_norm(nullptr, N, rank, &bytes);
    return bytes;
}

template <typename T>
static int normalize_impl(const T* Fd, int64_t ldf, int64_t N, int rank, double* dtil, double* qtil, double* A,
                          double* C, const NormWs& w, cudaStream_t s) {
    constexpr int VV = 16 / sizeof(T);   // rows per 16-byte vector
    const bool vec = (reinterpret_cast<uintptr_t>(Fd) % 16 == 0) && ((ldf * (int64_t)sizeof(T)) % 16 == 0);
    const int ncs = colsum_splits(N);
    const int64_t quantum = 32 * VV * 4;
    const int64_t per = ((N + ncs - 1) / ncs + quantum - 1) / quantum * quantum;
    const dim3 gcs((rank + 7) / 8, ncs);
    const unsigned rows_blocks = (unsigned)((N + 255) / 256);
    const unsigned vrows_blocks = (unsigned)((N + 256 * VV - 1) / (256 * VV));
    const size_t vsm = (size_t)rank * sizeof(double);
    if (vsm > 48 * 1024) {
        KEVD_CUDA_TRY(cudaFuncSetAttribute(k_rowdot<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
        KEVD_CUDA_TRY(cudaFuncSetAttribute(k_rowdot<T, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
    }

    KEVD_CUDA_TRY(cudaMemsetAsync(w.flags, 0, sizeof(int), s));
    {
        TraceScope tr(kStDegree, s);
        for (int pass = 0; pass < 2; ++pass) {
            const double* wdiv = pass == 0 ? nullptr : w.wa;   // 1/d~ for the second pass
            if (pass == 1) k_recip<<<rows_blocks, 256, 0, s>>>(dtil, N, w.wa);
            double* vec_out = pass == 0 ? w.svec : w.tvec;
            double* row_out = pass == 0 ? dtil : qtil;
            if (vec) k_colsum_partial<T, VV><<<gcs, 256, 0, s>>>(Fd, ldf, N, rank, per, wdiv, w.part);
            else k_colsum_partial<T, 1><<<gcs, 256, 0, s>>>(Fd, ldf, N, rank, per, wdiv, w.part);
            k_colsum_final<<<(rank + 255) / 256, 256, 0, s>>>(w.part, ncs, rank, vec_out);
            if (vec) k_rowdot<T, VV><<<vrows_blocks, 256, vsm, s>>>(Fd, ldf, N, rank, vec_out, row_out, w.flags, 1 << pass);
            else k_rowdot<T, 1><<<rows_blocks, 256, vsm, s>>>(Fd, ldf, N, rank, vec_out, row_out, w.flags, 1 << pass);
        }
    }
    KEVD_LAUNCH_CHECK();

    const int nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
    const int ns = gram_splits(N, ntri);
    {
        TraceScope tr(kStGram, s);
        k_gram_weights<<<rows_blocks, 256, 0, s>>>(dtil, qtil, N, w.wa, w.wc, w.waf, w.wcf);
        // FP32 F: FFMA products with round-to-nearest FP32 sums per row split.
        // (Tensor-core split products were measured to bias these N-long sums:
        // the MMA's FP32 accumulation truncates on every add.)
        if constexpr (std::is_same<T, float>::value)
            k_gram<T, float><<<dim3(ntri, ns), 256, 0, s>>>(Fd, ldf, N, rank, w.waf, w.wcf, w.gpart, nb, ntri);
        else
            k_gram<T, double><<<dim3(ntri, ns), 256, 0, s>>>(Fd, ldf, N, rank, w.wa, w.wc, w.gpart, nb, ntri);
    }
    {
        TraceScope tr(kStOther, s);
        k_gram_final<<<ntri, 256, 0, s>>>(w.gpart, ns, ntri, nb, rank, A, C);
    }
    KEVD_LAUNCH_CHECK();
    int flags = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&flags, w.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    if (flags & 4) return KEVD_ETIMEOUT;
    if (flags & 1) return KEVD_ED_NONPOS;
    if (flags & 2) return KEVD_EQ_NONPOS;
    return KEVD_OK;
}

extern "C" int bistoch_normalize(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf,
                                 double* dtil, double* qtil, double* A, double* C, void* workspace,
                                 size_t ws_bytes, void* stream) {
    if (!F || !dtil || !qtil || !A || !C) return KEVD_EINVAL;
    if (N < 1 || rank < 1 || rank > N || ldf < N || (f_dtype != KEVD_F64 && f_dtype != KEVD_F32)) return KEVD_EINVAL;
    size_t need = 0;
    NormWs w = carve_norm(workspace, N, rank, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (f_dtype == KEVD_F32)
        return normalize_impl(static_cast<const float*>(F), ldf, N, rank, dtil, qtil, A, C, w, s);
    return normalize_impl(static_cast<const double*>(F), ldf, N, rank, dtil, qtil, A, C, w, s);
}

// ---------------------------------------------------------------------------
// Symmetric normalisation (Section 2.1): d~ = F F^T 1 and the one Gram
// A_s = F^T D~^-1 F = (D~^-1/2 F)^T (D~^-1/2 F), whose eigenpairs give those of
// L~ = (D~^-1/2 F)(D~^-1/2 F)^T (the SVD form of the C = I case).
// ---------------------------------------------------------------------------
namespace kevd {
template <typename T>
static int symmetric_impl(const T* Fd, int64_t ldf, int64_t N, int rank, double* dtil, double* As, const NormWs& w,
                          cudaStream_t s) {
    constexpr int VV = 16 / sizeof(T);
    const bool vec = (reinterpret_cast<uintptr_t>(Fd) % 16 == 0) && ((ldf * (int64_t)sizeof(T)) % 16 == 0);
    const int ncs = colsum_splits(N);
    const int64_t quantum = 32 * VV * 4;
    const int64_t per = ((N + ncs - 1) / ncs + quantum - 1) / quantum * quantum;
    const dim3 gcs((rank + 7) / 8, ncs);
    const unsigned rows_blocks = (unsigned)((N + 255) / 256);
    const unsigned vrows_blocks = (unsigned)((N + 256 * VV - 1) / (256 * VV));
    const size_t vsm = (size_t)rank * sizeof(double);
    if (vsm > 48 * 1024) {
        KEVD_CUDA_TRY(cudaFuncSetAttribute(k_rowdot<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
        KEVD_CUDA_TRY(cudaFuncSetAttribute(k_rowdot<T, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));
    }
    KEVD_CUDA_TRY(cudaMemsetAsync(w.flags, 0, sizeof(int), s));
    {
        TraceScope tr(kStDegree, s);
        if (vec) k_colsum_partial<T, VV><<<gcs, 256, 0, s>>>(Fd, ldf, N, rank, per, nullptr, w.part);
        else k_colsum_partial<T, 1><<<gcs, 256, 0, s>>>(Fd, ldf, N, rank, per, nullptr, w.part);
        k_colsum_final<<<(rank + 255) / 256, 256, 0, s>>>(w.part, ncs, rank, w.svec);
        if (vec) k_rowdot<T, VV><<<vrows_blocks, 256, vsm, s>>>(Fd, ldf, N, rank, w.svec, dtil, w.flags, 1);
        else k_rowdot<T, 1><<<rows_blocks, 256, vsm, s>>>(Fd, ldf, N, rank, w.svec, dtil, w.flags, 1);
    }
    const int nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
    const int ns = gram_splits(N, ntri);
    {
        TraceScope tr(kStGram, s);
        k_recip<<<rows_blocks, 256, 0, s>>>(dtil, N, w.wa);
        if constexpr (std::is_same<T, float>::value) {
            k_recip_f<<<rows_blocks, 256, 0, s>>>(dtil, N, w.waf);
            k_gram<T, float><<<dim3(ntri, ns), 256, 0, s>>>(Fd, ldf, N, rank, w.waf, (const float*)nullptr, w.gpart, nb,
                                                            ntri);
        } else {
            k_gram<T, double><<<dim3(ntri, ns), 256, 0, s>>>(Fd, ldf, N, rank, w.wa, (const double*)nullptr, w.gpart,
                                                             nb, ntri);
        }
    }
    {
        TraceScope tr(kStOther, s);
        k_gram_final<<<ntri, 256, 0, s>>>(w.gpart, ns, ntri, nb, rank, As, nullptr);
    }
    KEVD_LAUNCH_CHECK();
    int flags = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&flags, w.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    return (flags & 1) ? KEVD_ED_NONPOS : KEVD_OK;
}
}  // namespace kevd

extern "C" int symmetric_normalize(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf, double* dtil,
                                   double* As, void* workspace, size_t ws_bytes, void* stream) {
    if (!F || !dtil || !As) return KEVD_EINVAL;
    if (N < 1 || rank < 1 || rank > N || ldf < N || (f_dtype != KEVD_F64 && f_dtype != KEVD_F32)) return KEVD_EINVAL;
    size_t need = 0;
    NormWs w = carve_norm(workspace, N, rank, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (f_dtype == KEVD_F32)
        return symmetric_impl(static_cast<const float*>(F), ldf, N, rank, dtil, As, w, s);
    return symmetric_impl(static_cast<const double*>(F), ldf, N, rank, dtil, As, w, s);
}

// Unweighted FP64 Gram G = U^T U of an N x k matrix (ld = ldu) through the same
// split kernel; gpart must hold gram_splits x ntri x 2 x 64 x 64 doubles.
size_t kevd_gram_partial_doubles(int64_t N, int k) {
    const int nb = (k + kevd::kGT - 1) / kevd::kGT, ntri = nb * (nb + 1) / 2;
    return (size_t)kevd::gram_splits(N, ntri) * ntri * 2 * kevd::kGT * kevd::kGT;
}

cudaError_t kevd_gram_plain(const double* U, int64_t ldu, int64_t N, int k, double* G, double* gpart, cudaStream_t s) {
    using namespace kevd;
    const int nb = (k + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
    const int ns = gram_splits(N, ntri);
    k_gram<double, double><<<dim3(ntri, ns), 256, 0, s>>>(U, ldu, N, k, (const double*)nullptr, (const double*)nullptr,
                                                          gpart, nb, ntri);
    k_gram_final<<<ntri, 256, 0, s>>>(gpart, ns, ntri, nb, k, G, nullptr);
    return cudaGetLastError();
}
