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
#include "gram_tc.cuh"
#include "tc_ptx.cuh"
#include "trace.cuh"

namespace kevd {

constexpr int kGT = 64;   // Gram output tile
constexpr int kGK = 16;   // rows per staged chunk

struct NormWs {
    double* part;   // ncs x rank column-sum partials
    double* svec;   // rank
    double* tvec;   // rank
    int* flags;     // bit 0: some d~ <= 0, bit 1: some q~ <= 0
    double* wa;     // N rounded up to 64: 1 / d~_i^2, zero past N
    double* wc;     // N rounded up to 64: 1 / q~_i, zero past N
    float* waf;     // N rounded up to 64: FP32 copies of the Gram weights (FP32 path), zero past N
    float* wcf;
    unsigned* cmax; // 3 x rank: column maxima of |F|, |wa F|, |wc F| (tensor-core Gram, FP32 F)
    float* mag;     // 3 x rank: their grid magic numbers
    unsigned long long* cmax64;   // 3 x rank: the same maxima for FP64 F
    int* ecol;      // 3 x rank: their exponents
    uint16_t* planes;   // FP64 Gram: digit planes of one slab of rows
    double* gpart;  // nsplit x ntri x 2 x 64 x 64 Gram partials (128 x 128 for FP32 F)
};

constexpr int kSMs = 152;   // wave sizing of the Gram grids (a performance choice only)

static int colsum_splits(int64_t N) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 4096)); }

static int gram_splits(int64_t N, int64_t ntri) {
    int64_t s = (1216 + ntri - 1) / ntri;
    s = std::min<int64_t>(s, std::max<int64_t>(1, N / 512));
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, 64));
}

// Row split of the 128-tile FP32 Gram: `per` rows (a multiple of 32, at least
// 1,024 unless N is smaller) per CTA, the split count chosen so that
// ntri x nsplit CTAs fill whole waves of one CTA per SM (152 SMs); a larger
// split count is taken only when it raises the wave efficiency by > 2%.
constexpr int kG2Tile = 128;
static int64_t gram32_per(int64_t N, int64_t ntri, int* nsplit) {
    int64_t best_per = (N + 31) / 32 * 32;
    double best_eff = -1.0;
    for (int64_t sp = 1; sp <= 64; ++sp) {
        const int64_t per = ((N + sp - 1) / sp + 31) / 32 * 32;
        if (sp > 1 && per < 1024) break;
        const int64_t ns = (N + per - 1) / per, blocks = ntri * ns;
        const double eff = (double)blocks / (double)(((blocks + kSMs - 1) / kSMs) * kSMs);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best_per = per;
        }
    }
    *nsplit = (int)((N + best_per - 1) / best_per);
    return best_per;
}

// fp64: room for the digit planes of the FP64 factor's tensor-core Grams.
static NormWs carve_norm(void* base, int64_t N, int rank, size_t* bytes, bool fp64) {
    Carver c(base);
    const int64_t nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
    const int64_t nb2 = (rank + kG2Tile - 1) / kG2Tile, ntri2 = nb2 * (nb2 + 1) / 2;
    int ns2 = 1, ns3 = 1;
    gram32_per(N, ntri2, &ns2);
    gram_tc_per(N, ntri2, kSMs, &ns3);
    const size_t gp64 = (size_t)gram_splits(N, ntri) * ntri * 2 * kGT * kGT;
    const size_t gp32 = (size_t)std::max(ns2, ns3) * ntri2 * 2 * kG2Tile * kG2Tile;
    const size_t gpoz = std::max(gram_oz_partial_doubles(N, rank, 2, kSMs), gram_oz_partial_doubles(N, rank, 1, kSMs));
    const int64_t Npad = (N + 63) / 64 * 64;
    NormWs w;
    w.part = c.take<double>((size_t)colsum_splits(N) * rank);
    w.svec = c.take<double>(rank);
    w.tvec = c.take<double>(rank);
    w.flags = c.take<int>(4);
    w.wa = c.take<double>(Npad);
    w.wc = c.take<double>(Npad);
    w.waf = c.take<float>(Npad);
    w.wcf = c.take<float>(Npad);
    w.cmax = c.take<unsigned>(3 * (size_t)rank);
    w.mag = c.take<float>(3 * (size_t)rank);
    w.cmax64 = c.take<unsigned long long>(3 * (size_t)rank);
    w.ecol = c.take<int>(3 * (size_t)rank);
    w.gpart = c.take<double>(std::max(std::max(gp64, gp32), gpoz));
    w.planes = fp64 ? c.take<uint16_t>(std::max(gram_oz_plane_bytes(N, rank, 2), gram_oz_plane_bytes(N, rank, 1)) / 2)
                    : nullptr;
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
                                                        int64_t per, const T* __restrict__ wmul,
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
        VT x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = *reinterpret_cast<const VT*>(col + i + u * STEP);
        if (wmul) {
#pragma unroll
            for (int u = 0; u < 4; ++u) y[u] = *reinterpret_cast<const VT*>(wmul + i + u * STEP);
        }
        T blk = T(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T* e = reinterpret_cast<const T*>(&x[u]);
            const T* f = reinterpret_cast<const T*>(&y[u]);
#pragma unroll
            for (int q = 0; q < V; ++q) blk += wmul ? e[q] * f[q] : e[q];
        }
        acc += (double)blk;
    }
    for (; i < i1; i += STEP)
        for (int q = 0; q < V && i + q < i1; ++q) acc += (double)(wmul ? col[i + q] * wmul[i + q] : col[i + q]);
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

// As k_recip, and zero for N <= i < Npad.
__global__ void k_recip_pad(const double* __restrict__ x, int64_t N, int64_t Npad, double* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] = 1.0 / x[i];
    else if (i < Npad) y[i] = 0.0;
}

// y_i = 1/x_i in FP32 for i < N, 0 for N <= i < Npad (the zero padding the
// tensor-core Gram's weight copies read).
__global__ void k_recip_f(const double* __restrict__ x, int64_t N, int64_t Npad, float* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] = (float)(1.0 / x[i]);
    else if (i < Npad) y[i] = 0.f;
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

// Row weights of the two Grams: 1/d~^2 and 1/q~ (one division each per row);
// all four arrays are zero for N <= i < Npad.
__global__ void k_gram_weights(const double* __restrict__ dtil, const double* __restrict__ qtil, int64_t N,
                               int64_t Npad, double* __restrict__ wa, double* __restrict__ wc,
                               float* __restrict__ waf, float* __restrict__ wcf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) {
        if (i < Npad) {
            wa[i] = wc[i] = 0.0;
            waf[i] = wcf[i] = 0.f;
        }
        return;
    }
    const double d = dtil[i];
    wa[i] = 1.0 / (d * d);
    wc[i] = 1.0 / qtil[i];
    waf[i] = (float)wa[i];
    wcf[i] = (float)wc[i];
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

// FP32 weighted Grams, 128 x 128 output tiles (one CTA per SM: 256 threads,
// up to 128 FP32 accumulators each).  Thread (tx, ty) owns rows
// {4ty..4ty+3, 64+4ty..64+4ty+3} x cols {4tx..4tx+3, 64+4tx..64+4tx+3} of each
// Gram, so every k step is 2 (Ua) + 2 (Uc) + 2 (V) 16-byte shared loads for 128
// FFMAs.  Rows are consumed in chunks of 16:
//   * asynchronous copies (cp.async, 16 bytes along n; 4 bytes when F or ldf
//     is not 16-byte aligned) bring F(r:r+16, I-block), F(r:r+16, J-block) and
//     the two weight vectors into a raw staging buffer two chunks ahead, with
//     zero fill past the split's last row and past `rank`;
//   * the raw chunk is then scaled by the weights and stored transposed
//     (k-major) with the column index XOR-ed by 8 * (k >> 2), so the transposed
//     stores hit 32 distinct banks and the 16-byte k-step loads stay contiguous
//     and conflict-free;
//   * the FFMAs of chunk c run while the copies of chunk c + 2 are in flight.
// Sums are FP32 with round-to-nearest over one row split of `per` rows (a
// multiple of 32); k_gram_final adds the splits in FP64.
constexpr int kG2T = 128;   // output tile
constexpr int kG2K = 16;    // rows per chunk

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// QM: quadrant mask of the tile, bit 0 rows 0-63 x cols 64-127, bit 1 rows
// 64-127 x cols 0-63, bit 2 rows 64-127 x cols 64-127 (rows 0-63 x cols 0-63
// always).  Quadrants off the mask are not formed: rows or cols past rank,
// and the strictly lower quadrant of a diagonal tile (never read by
// k_gram_final).
template <bool TWO, int QM>
__device__ __forceinline__ void gram32_body(const float* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                            const float* __restrict__ wa, const float* __restrict__ wc,
                                            double* __restrict__ gpart, int I, int J, int ntri, int64_t per,
                                            int vec) {
    constexpr bool q01 = (QM & 1) != 0, q10 = (QM & 2) != 0, q11 = (QM & 4) != 0;
    constexpr int NU = TWO ? 3 : 2;                // Ua, (Uc), V
    constexpr int kPlane = kG2K * kG2T;            // floats per transposed operand
    constexpr int kT = NU * kPlane;                // one transposed stage
    constexpr int kRaw = 2 * kG2T * kG2K + 2 * kG2K;   // raw F(I), F(J) [col][row], wa, wc
    extern __shared__ float4 g32_smem[];
    float* sm = reinterpret_cast<float*>(g32_smem);
    float* tbuf = sm;                 // 2 x kT
    float* raw = sm + 2 * kT;         // 2 x kRaw
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const int nchunks = i1 > i0 ? (int)((i1 - i0 + kG2K - 1) / kG2K) : 0;

    // copy / transpose mapping: e = tid + 256 p (p = 0..1): column e >> 2 of
    // the block, row quad e & 3 of the chunk (the same quad for both p)
    const int kq = tid & 3;
    auto issue = [&](int ch) {
        float* rb = raw + (ch & 1) * kRaw;
        const int64_t r = i0 + (int64_t)ch * kG2K + 4 * kq;
        const int64_t left = i1 - r;                 // rows of this quad inside the split
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int col = (tid + 256 * p) >> 2;
#pragma unroll
            for (int blk = 0; blk < 2; ++blk) {
                const int c = (blk == 0 ? I : J) * kG2T + col;
                const uint32_t dst = smem_u32(rb + (blk * kG2T + col) * kG2K + 4 * kq);
                const bool ok = c < rank && left > 0;
                const float* src = ok ? F + (int64_t)c * ldf + r : F;
                if (vec) {
                    cp_async16(dst, src, ok ? (uint32_t)(4 * (left < 4 ? left : 4)) : 0u);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool in = ok && q < left;
                        cp_async4(dst + 4 * q, in ? src + q : F, in ? 4u : 0u);
                    }
                }
            }
        }
        if (tid < 8) {   // weights: threads 0..3 wa, 4..7 wc (quad tid & 3)
            const float* wv = tid < 4 ? wa : (TWO ? wc : wa);
            const uint32_t dst = smem_u32(rb + 2 * kG2T * kG2K + (tid >> 2) * kG2K + 4 * kq);
            const bool ok = left > 0;
            if (vec) {
                cp_async16(dst, ok ? wv + r : wv, ok ? (uint32_t)(4 * (left < 4 ? left : 4)) : 0u);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const bool in = ok && q < left;
                    cp_async4(dst + 4 * q, in ? wv + r + q : wv, in ? 4u : 0u);
                }
            }
        }
    };
    auto transpose = [&](int ch) {
        const float* rb = raw + (ch & 1) * kRaw;
        float* ua = tbuf + (ch & 1) * kT;
        float* uc = ua + kPlane;
        float* v = ua + (NU - 1) * kPlane;
        const float4 w4 = *reinterpret_cast<const float4*>(rb + 2 * kG2T * kG2K + 4 * kq);
        const float4 c4 = *reinterpret_cast<const float4*>(rb + 2 * kG2T * kG2K + kG2K + 4 * kq);
        const float wq[4] = {w4.x, w4.y, w4.z, w4.w}, cq[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int col = (tid + 256 * p) >> 2;
            const int sc = col ^ (kq << 3);
            const float4 fi = *reinterpret_cast<const float4*>(rb + col * kG2K + 4 * kq);
            const float4 fj = *reinterpret_cast<const float4*>(rb + (kG2T + col) * kG2K + 4 * kq);
            const float fi4[4] = {fi.x, fi.y, fi.z, fi.w}, fj4[4] = {fj.x, fj.y, fj.z, fj.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int o = (4 * kq + q) * kG2T + sc;
                ua[o] = fi4[q] * wq[q];
                if (TWO) uc[o] = fi4[q] * cq[q];
                v[o] = fj4[q];
            }
        }
    };

    float aa[8][8], ac[TWO ? 8 : 1][TWO ? 8 : 1];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            aa[a][c] = 0.f;
            if (TWO) ac[TWO ? a : 0][TWO ? c : 0] = 0.f;
        }

    // prologue: chunks 0 and 1 in flight, chunk 0 transposed
    if (nchunks > 0) issue(0);
    cp_async_commit();
    if (nchunks > 1) issue(1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    if (nchunks > 0) transpose(0);
    __syncthreads();
    for (int ch = 0; ch < nchunks; ++ch) {
        if (ch + 2 < nchunks) issue(ch + 2);   // into the raw buffer chunk ch left
        cp_async_commit();                     // (an empty group keeps the count uniform)
        const float* ua = tbuf + (ch & 1) * kT;
        const float* uc = ua + kPlane;
        const float* v = ua + (NU - 1) * kPlane;
#pragma unroll 1
        for (int g = 0; g < kG2K / 4; ++g) {
            const int ra = (ty << 2) ^ (g << 3), rv = (tx << 2) ^ (g << 3);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = 4 * g + q;
                const float4 a0 = *reinterpret_cast<const float4*>(ua + kk * kG2T + ra);
                const float4 a1 = *reinterpret_cast<const float4*>(ua + kk * kG2T + 64 + ra);
                const float4 v0 = *reinterpret_cast<const float4*>(v + kk * kG2T + rv);
                const float4 v1 = *reinterpret_cast<const float4*>(v + kk * kG2T + 64 + rv);
                const float a8[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float v8[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (a < 4 ? (c < 4 || q01) : (c < 4 ? q10 : q11)) aa[a][c] = fmaf(a8[a], v8[c], aa[a][c]);
                if (TWO) {
                    const float4 c0 = *reinterpret_cast<const float4*>(uc + kk * kG2T + ra);
                    const float4 c1 = *reinterpret_cast<const float4*>(uc + kk * kG2T + 64 + ra);
                    const float c8[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                    for (int a = 0; a < 8; ++a)
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (a < 4 ? (c < 4 || q01) : (c < 4 ? q10 : q11))
                                ac[TWO ? a : 0][TWO ? c : 0] = fmaf(c8[a], v8[c], ac[TWO ? a : 0][TWO ? c : 0]);
                }
            }
        }
        if (ch + 1 < nchunks) {
            cp_async_wait1();   // chunk ch + 1 landed (only chunk ch + 2 may be pending)
            __syncthreads();
            transpose(ch + 1);
        }
        __syncthreads();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");

    double* out = gpart + ((size_t)blockIdx.y * ntri + blockIdx.x) * 2 * kG2T * kG2T;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int row = (a < 4 ? 0 : 64) + 4 * ty + (a & 3);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = 64 * h + 4 * tx;
            double2* o = reinterpret_cast<double2*>(out + row * kG2T + col);
            o[0] = make_double2(aa[a][4 * h], aa[a][4 * h + 1]);
            o[1] = make_double2(aa[a][4 * h + 2], aa[a][4 * h + 3]);
            if (TWO) {   // the second Gram's half is neither written nor read when only one is formed
                double2* oc = reinterpret_cast<double2*>(out + kG2T * kG2T + row * kG2T + col);
                oc[0] = make_double2(ac[TWO ? a : 0][TWO ? 4 * h : 0], ac[TWO ? a : 0][TWO ? 4 * h + 1 : 0]);
                oc[1] = make_double2(ac[TWO ? a : 0][TWO ? 4 * h + 2 : 0], ac[TWO ? a : 0][TWO ? 4 * h + 3 : 0]);
            }
        }
    }
}

template <bool TWO>
__global__ void __launch_bounds__(256, 1) k_gram32(const float* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                                   const float* __restrict__ wa, const float* __restrict__ wc,
                                                   double* __restrict__ gpart, int nb, int ntri, int64_t per,
                                                   int vec) {
    int I, J;
    tri_decode(blockIdx.x, nb, I, J);
    const bool rhi = I * kG2T + 64 < rank, chi = J * kG2T + 64 < rank;
    const int qm = (chi ? 1 : 0) | (rhi && I != J ? 2 : 0) | (rhi && chi ? 4 : 0);
    // I <= J: rhi is false only on the last block row (then I == J), chi only on
    // the last block column, so the mask is 7 (interior), 5 (diagonal), 2 (last
    // block column, 64 or fewer columns left) or 0 (last diagonal tile, ditto)
    if (qm == 5) gram32_body<TWO, 5>(F, ldf, N, rank, wa, wc, gpart, I, J, ntri, per, vec);
    else if (qm == 2) gram32_body<TWO, 2>(F, ldf, N, rank, wa, wc, gpart, I, J, ntri, per, vec);
    else if (qm == 0) gram32_body<TWO, 0>(F, ldf, N, rank, wa, wc, gpart, I, J, ntri, per, vec);
    else gram32_body<TWO, 7>(F, ldf, N, rank, wa, wc, gpart, I, J, ntri, per, vec);
}

// Sum the split partials in order; write (I-row a, J-col c) and its mirror.
// Diagonal tiles keep their upper triangle only, so A and C are exactly symmetric.
// ACC adds the sums to A and C instead (each entry has one owner thread, and a
// diagonal entry is added once).
// P: element type of the partials (FP64, or FP32 from the tensor-core kernel).
template <int TT, bool ACC = false, typename P = double>
__global__ void k_gram_final(const P* __restrict__ gpart, int nsplit, int ntri, int nb, int rank,
                             double* __restrict__ A, double* __restrict__ C) {
    const int t = blockIdx.x;
    int I, J;
    tri_decode(t, nb, I, J);
    for (int e = threadIdx.x; e < TT * TT; e += blockDim.x) {
        const int a = e / TT, c = e % TT;
        const int ra = I * TT + a, rc = J * TT + c;
        if (ra >= rank || rc >= rank) continue;
        if (I == J && a > c) continue;
        double sa = 0.0, sc = 0.0;
        for (int q = 0; q < nsplit; ++q) {
            const P* p = gpart + ((size_t)q * ntri + t) * 2 * TT * TT;
            sa += (double)p[e];
            if (C) sc += (double)p[TT * TT + e];
        }
        if (ACC) {
            A[(int64_t)rc * rank + ra] += sa;
            if (ra != rc) A[(int64_t)ra * rank + rc] += sa;
            if (C) {
                C[(int64_t)rc * rank + ra] += sc;
                if (ra != rc) C[(int64_t)ra * rank + rc] += sc;
            }
            continue;
        }
        A[(int64_t)rc * rank + ra] = sa;
        A[(int64_t)ra * rank + rc] = sa;
        if (C) {
            C[(int64_t)rc * rank + ra] = sc;
            C[(int64_t)ra * rank + rc] = sc;
        }
    }
}

// FP32 F: the tensor-core Gram kernel (gram_tc.cu) when the tensor map can
// describe F, else the 128-tile FFMA kernel; then the FP64 sum over row
// splits.  wc == nullptr forms the first Gram only (C is not written).
static cudaError_t gram32(const float* F, int64_t ldf, int64_t N, int rank, const float* wa, const float* wc,
                          double* gpart, double* A, double* C, const NormWs& w, cudaStream_t s) {
    const int nb = (rank + kG2T - 1) / kG2T, ntri = nb * (nb + 1) / 2;
    if (gram_tc_eligible(F, ldf, N, rank)) {
        int ns = 1;
        const int64_t per = gram_tc_per(N, ntri, kSMs, &ns);
        {
            TraceScope tr(kStGram, s);
            float* gp32 = reinterpret_cast<float*>(gpart);
            cudaError_t e = launch_gram_tc(F, ldf, N, rank, wa, wc, w.cmax, w.mag, gp32, w.flags, nb, ntri, per, ns, s);
            if (e != cudaSuccess) return e;
        }
        {
            TraceScope tr(kStOther, s);
            k_gram_final<kG2T, false, float><<<ntri, 256, 0, s>>>(reinterpret_cast<const float*>(gpart), ns, ntri, nb,
                                                                  rank, A, C);
        }
        return cudaGetLastError();
    }
    int ns = 1;
    const int64_t per = gram32_per(N, ntri, &ns);
    const int vec = (reinterpret_cast<uintptr_t>(F) % 16 == 0) && (ldf % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(wa) % 16 == 0) && (!wc || reinterpret_cast<uintptr_t>(wc) % 16 == 0);
    const dim3 grid(ntri, ns);
    {
        TraceScope tr(kStGram, s);
        if (wc) {
            const int smem = (2 * 3 * kG2K * kG2T + 2 * (2 * kG2T * kG2K + 2 * kG2K)) * (int)sizeof(float);
            cudaError_t e = cudaFuncSetAttribute(k_gram32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            k_gram32<true><<<grid, 256, smem, s>>>(F, ldf, N, rank, wa, wc, gpart, nb, ntri, per, vec);
        } else {
            const int smem = (2 * 2 * kG2K * kG2T + 2 * (2 * kG2T * kG2K + 2 * kG2K)) * (int)sizeof(float);
            cudaError_t e = cudaFuncSetAttribute(k_gram32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            k_gram32<false><<<grid, 256, smem, s>>>(F, ldf, N, rank, wa, nullptr, gpart, nb, ntri, per, vec);
        }
    }
    {
        TraceScope tr(kStOther, s);
        k_gram_final<kG2T><<<ntri, 256, 0, s>>>(gpart, ns, ntri, nb, rank, A, C);
    }
    return cudaGetLastError();
}

}  // namespace kevd

using namespace kevd;

size_t kevd_normalize_ws(int64_t N, int32_t rank, bool fp64) {
    if (N < 1 || rank < 1) return 0;
    size_t bytes = 0;
    carve_norm(nullptr, N, rank, &bytes, fp64);
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
            // 1/d~ for the second pass, in F's type (the FP32 sums multiply in FP32): converted
            // once per row here, not once per element in each of the rank columns
            const T* wdiv = nullptr;
            if (pass == 1) {
                if constexpr (std::is_same<T, float>::value) {
                    k_recip_f<<<rows_blocks, 256, 0, s>>>(dtil, N, N, w.waf);
                    wdiv = w.waf;
                } else {
                    k_recip<<<rows_blocks, 256, 0, s>>>(dtil, N, w.wa);
                    wdiv = w.wa;
                }
            }
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

    {
        TraceScope tr(kStGram, s);
        const int64_t Npad = (N + 63) / 64 * 64;
        k_gram_weights<<<(unsigned)((Npad + 255) / 256), 256, 0, s>>>(dtil, qtil, N, Npad, w.wa, w.wc, w.waf, w.wcf);
    }
    if constexpr (std::is_same<T, float>::value) {
        // FP32 F: tensor-core slice products with the leading product summed
        // exactly (plain split products in the MMA's FP32 accumulation were
        // measured to bias these N-long sums), or the FFMA kernel.
        KEVD_CUDA_TRY(gram32(Fd, ldf, N, rank, w.waf, w.wcf, w.gpart, A, C, w, s));
    } else if (gram_oz_eligible(reinterpret_cast<const double*>(Fd), ldf, N, rank)) {
        // FP64 F: digit-sliced products on the tensor cores at FP64 accuracy
        TraceScope tr(kStGram, s);
        KEVD_CUDA_TRY(launch_gram_oz(reinterpret_cast<const double*>(Fd), ldf, N, rank, w.wa, w.wc, w.waf, w.wcf,
                                     w.cmax64, w.ecol,
                                     w.gpart, w.planes, w.flags, A, C, kSMs, s));
    } else {
        const int nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
        const int ns = gram_splits(N, ntri);
        {
            TraceScope tr(kStGram, s);
            k_gram<T, double><<<dim3(ntri, ns), 256, 0, s>>>(Fd, ldf, N, rank, w.wa, w.wc, w.gpart, nb, ntri);
        }
        {
            TraceScope tr(kStOther, s);
            k_gram_final<kGT><<<ntri, 256, 0, s>>>(w.gpart, ns, ntri, nb, rank, A, C);
        }
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
    NormWs w = carve_norm(workspace, N, rank, &need, f_dtype == KEVD_F64);
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
    {
        TraceScope tr(kStGram, s);
        const int64_t Npad = (N + 63) / 64 * 64;
        k_recip_pad<<<(unsigned)((Npad + 255) / 256), 256, 0, s>>>(dtil, N, Npad, w.wa);
        if constexpr (std::is_same<T, float>::value)
            k_recip_f<<<(unsigned)((Npad + 255) / 256), 256, 0, s>>>(dtil, N, Npad, w.waf);
    }
    if constexpr (std::is_same<T, float>::value) {
        KEVD_CUDA_TRY(gram32(Fd, ldf, N, rank, w.waf, nullptr, w.gpart, As, nullptr, w, s));
    } else if (gram_oz_eligible(reinterpret_cast<const double*>(Fd), ldf, N, rank)) {
        TraceScope tr(kStGram, s);
        KEVD_CUDA_TRY(launch_gram_oz(reinterpret_cast<const double*>(Fd), ldf, N, rank, w.wa, nullptr, w.waf, w.wcf,
                                     w.cmax64, w.ecol, w.gpart, w.planes, w.flags, As, nullptr, kSMs, s));
    } else {
        const int nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
        const int ns = gram_splits(N, ntri);
        {
            TraceScope tr(kStGram, s);
            k_gram<T, double><<<dim3(ntri, ns), 256, 0, s>>>(Fd, ldf, N, rank, w.wa, (const double*)nullptr, w.gpart,
                                                             nb, ntri);
        }
        {
            TraceScope tr(kStOther, s);
            k_gram_final<kGT><<<ntri, 256, 0, s>>>(w.gpart, ns, ntri, nb, rank, As, nullptr);
        }
    }
    KEVD_LAUNCH_CHECK();
    int flags = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&flags, w.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    if (flags & 4) return KEVD_ETIMEOUT;
    return (flags & 1) ? KEVD_ED_NONPOS : KEVD_OK;
}
}  // namespace kevd

extern "C" int symmetric_normalize(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf, double* dtil,
                                   double* As, void* workspace, size_t ws_bytes, void* stream) {
    if (!F || !dtil || !As) return KEVD_EINVAL;
    if (N < 1 || rank < 1 || rank > N || ldf < N || (f_dtype != KEVD_F64 && f_dtype != KEVD_F32)) return KEVD_EINVAL;
    size_t need = 0;
    NormWs w = carve_norm(workspace, N, rank, &need, f_dtype == KEVD_F64);
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
    k_gram_final<kGT><<<ntri, 256, 0, s>>>(gpart, ns, ntri, nb, k, G, nullptr);
    return cudaGetLastError();
}

// Weighted FP64 Grams A (+)= F^T diag(wa) F and C (+)= F^T diag(wc) F of an
// N x rank block of rows (ld = ldf), through the same split kernel; acc = 1
// adds to A and C (panel-by-panel accumulation), acc = 0 overwrites them.
// gpart must hold kevd_gram_partial_doubles(N, rank) doubles.
cudaError_t kevd_gram_weighted(const double* F, int64_t ldf, int64_t N, int rank, const double* wa, const double* wc,
                               double* gpart, double* A, double* C, int acc, cudaStream_t s) {
    using namespace kevd;
    const int nb = (rank + kGT - 1) / kGT, ntri = nb * (nb + 1) / 2;
    const int ns = gram_splits(N, ntri);
    k_gram<double, double><<<dim3(ntri, ns), 256, 0, s>>>(F, ldf, N, rank, wa, wc, gpart, nb, ntri);
    if (acc) k_gram_final<kGT, true><<<ntri, 256, 0, s>>>(gpart, ns, ntri, nb, rank, A, C);
    else k_gram_final<kGT, false><<<ntri, 256, 0, s>>>(gpart, ns, ntri, nb, rank, A, C);
    return cudaGetLastError();
}
