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
    double* gpart;  // nsplit x ntri x 2 x 64 x 64
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
    w.gpart = c.take<double>((size_t)gram_splits(N, ntri) * ntri * 2 * kGT * kGT);
    *bytes = c.off;
    return w;
}

// Partial column sums of F (weighted by 1/wdiv_i when wdiv != nullptr).
// Block: 8 warps = 8 columns; blockIdx.y = row split.
__global__ void k_colsum_partial(const double* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                 const double* __restrict__ wdiv, double* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= rank) return;
    const int64_t per = (N + gridDim.y - 1) / gridDim.y;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const double* col = F + (int64_t)c * ldf;
    double s = 0.0;
    if (wdiv) {
        for (int64_t i = i0 + lane; i < i1; i += 32) s += col[i] / wdiv[i];
    } else {
        for (int64_t i = i0 + lane; i < i1; i += 32) s += col[i];
    }
    s = warp_sum(s);
    if (lane == 0) part[(size_t)blockIdx.y * rank + c] = s;
}

__global__ void k_colsum_final(const double* __restrict__ part, int nsplit, int rank, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= rank) return;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += part[(size_t)q * rank + c];
    out[c] = s;
}

// out_i = F(i,:) . v ; flag bit if out_i <= 0 (or not a number).
__global__ void k_rowdot(const double* __restrict__ F, int64_t ldf, int64_t N, int rank,
                         const double* __restrict__ v, double* __restrict__ out, int* flags, int bit) {
    extern __shared__ double vs[];
    for (int c = threadIdx.x; c < rank; c += blockDim.x) vs[c] = v[c];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double s = 0.0;
    for (int c = 0; c < rank; ++c) s = fma(F[(int64_t)c * ldf + i], vs[c], s);
    out[i] = s;
    if (!(s > 0.0)) atomicOr(flags, bit);
}

// Row weights of the two Grams: 1/d~^2 and 1/q~ (one division each per row).
__global__ void k_gram_weights(const double* __restrict__ dtil, const double* __restrict__ qtil, int64_t N,
                               double* __restrict__ wa, double* __restrict__ wc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double d = dtil[i];
    wa[i] = 1.0 / (d * d);
    wc[i] = 1.0 / qtil[i];
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
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                              const double* __restrict__ wa, const double* __restrict__ wc,
                                              double* __restrict__ gpart, int nb, int ntri) {
    constexpr int P = kGT + 4;
    __shared__ __align__(16) double Ua[kGK][P];   // F(:,I) * wa
    __shared__ __align__(16) double Uc[kGK][P];   // F(:,I) * wc
    __shared__ __align__(16) double V[kGK][P];    // F(:,J)
    int I, J;
    tri_decode(blockIdx.x, nb, I, J);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t per = (N + gridDim.y - 1) / gridDim.y;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    double aa[4][4], ac[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) aa[a][c] = ac[a][c] = 0.0;

    for (int64_t r0 = i0; r0 < i1; r0 += kGK) {
#pragma unroll
        for (int p = 0; p < (kGK * kGT) / 256; ++p) {
            const int e = tid + 256 * p, kk = e % kGK, col = e / kGK;
            const int64_t row = r0 + kk;
            const int ci = I * kGT + col, cj = J * kGT + col;
            double fi = 0.0, fj = 0.0, a = 0.0, c = 0.0;
            if (row < i1) {
                if (ci < rank) fi = F[(int64_t)ci * ldf + row];
                if (cj < rank) fj = F[(int64_t)cj * ldf + row];
                a = wa[row];
                c = wc[row];
            }
            Ua[kk][col] = fi * a;
            Uc[kk][col] = fi * c;
            V[kk][col] = fj;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            const double2 ua0 = *reinterpret_cast<const double2*>(&Ua[kk][ty * 4]);
            const double2 ua1 = *reinterpret_cast<const double2*>(&Ua[kk][ty * 4 + 2]);
            const double2 uc0 = *reinterpret_cast<const double2*>(&Uc[kk][ty * 4]);
            const double2 uc1 = *reinterpret_cast<const double2*>(&Uc[kk][ty * 4 + 2]);
            const double2 v0 = *reinterpret_cast<const double2*>(&V[kk][tx * 4]);
            const double2 v1 = *reinterpret_cast<const double2*>(&V[kk][tx * 4 + 2]);
            const double a4[4] = {ua0.x, ua0.y, ua1.x, ua1.y};
            const double c4[4] = {uc0.x, uc0.y, uc1.x, uc1.y};
            const double v4[4] = {v0.x, v0.y, v1.x, v1.y};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    aa[a][c] = fma(a4[a], v4[c], aa[a][c]);
                    ac[a][c] = fma(c4[a], v4[c], ac[a][c]);
                }
        }
        __syncthreads();
    }
    double* out = gpart + ((size_t)blockIdx.y * ntri + blockIdx.x) * 2 * kGT * kGT;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            out[(ty * 4 + a) * kGT + tx * 4 + c] = aa[a][c];
            out[kGT * kGT + (ty * 4 + a) * kGT + tx * 4 + c] = ac[a][c];
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
        C[(int64_t)rc * rank + ra] = sc;
        C[(int64_t)ra * rank + rc] = sc;
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

extern "C" int bistoch_normalize(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf,
                                 double* dtil, double* qtil, double* A, double* C, void* workspace,
                                 size_t ws_bytes, void* stream) {
    if (!F || !dtil || !qtil || !A || !C) return KEVD_EINVAL;
    if (N < 1 || rank < 1 || rank > N || ldf < N || f_dtype != KEVD_F64) return KEVD_EINVAL;
    size_t need = 0;
    NormWs w = carve_norm(workspace, N, rank, &need);
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double* Fd = static_cast<const double*>(F);
    const int ncs = colsum_splits(N);
    const dim3 gcs((rank + 7) / 8, ncs);
    const unsigned rows_blocks = (unsigned)((N + 255) / 256);
    const size_t vsm = (size_t)rank * sizeof(double);
    if (vsm > 48 * 1024) KEVD_CUDA_TRY(cudaFuncSetAttribute(k_rowdot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vsm));

    KEVD_CUDA_TRY(cudaMemsetAsync(w.flags, 0, sizeof(int), s));
    {
        TraceScope tr(kStDegree, s);
        k_colsum_partial<<<gcs, 256, 0, s>>>(Fd, ldf, N, rank, nullptr, w.part);
        k_colsum_final<<<(rank + 255) / 256, 256, 0, s>>>(w.part, ncs, rank, w.svec);
        k_rowdot<<<rows_blocks, 256, vsm, s>>>(Fd, ldf, N, rank, w.svec, dtil, w.flags, 1);
        k_colsum_partial<<<gcs, 256, 0, s>>>(Fd, ldf, N, rank, dtil, w.part);
        k_colsum_final<<<(rank + 255) / 256, 256, 0, s>>>(w.part, ncs, rank, w.tvec);
        k_rowdot<<<rows_blocks, 256, vsm, s>>>(Fd, ldf, N, rank, w.tvec, qtil, w.flags, 2);
    }
    KEVD_LAUNCH_CHECK();

    const int nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
    const int ns = gram_splits(N, ntri);
    {
        TraceScope tr(kStGram, s);
        k_gram_weights<<<rows_blocks, 256, 0, s>>>(dtil, qtil, N, w.wa, w.wc);
        k_gram<<<dim3(ntri, ns), 256, 0, s>>>(Fd, ldf, N, rank, w.wa, w.wc, w.gpart, nb, ntri);
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
    if (flags & 1) return KEVD_ED_NONPOS;
    if (flags & 2) return KEVD_EQ_NONPOS;
    return KEVD_OK;
}
