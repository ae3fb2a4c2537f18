// FP64-accurate products C = A B^T on the tensor cores from precomputed digit
// planes, for the kernel-column engine of the FP64 path (Algorithm 2):
// X X(S,:)^T, F(:, :k) F(S, :k)^T and the solve G = R L^-T of each round.
//
// Operands.  A matrix enters as the seven-digit slicing of oz_digits.cuh with
// one exponent per row (max |row| < 2^E, so x = 2^(E - 6) sum_s d_s 2^(-8 s)
// up to 2^(E - 55)): plane s holds p_s = d_s 2^(-8 s) as BF16, K-major (the K
// values of a row contiguous, word pairs of consecutive K), planes[s plane +
// i ldk + c].  The producers (factor.cu) cut each operand once: X at the start
// of the factorisation, F's new columns in the epilogue of the solve (rows of
// F have norm <= 1 for the Gaussian kernel, so one exponent, E = 1, serves
// every row and the planes of old columns never change), R and L^-1 once per
// round, the pivot panels as gathers of rows of the X and F planes.  Columns
// past K up to the next multiple of 16 are zero in both operands.
//
// Products.  The 28 digit pairs with s + t <= 6 are formed; levels 0-3 and the
// two halves of level 4 sum exactly in FP32 TMEM accumulators over 256-column
// chunks, levels 5-6 in a seventh (see ozgemm.cu); after each chunk the exact
// levels go into an INT64 running sum (units 2^-24) and the rest into an FP32
// one.  C(i, j) = 2^(E_i + E_j - 36) (T + M 2^24).
//
// Tiles: M = 128 rows of A by N = 64 rows of B (128 for three digits, whose
// three accumulators leave TMEM room for the wider shape), the contraction in
// 16-column quarters through a TMA ring (one 3-D load of 16 columns x 128 rows x
// D planes of A and one of B per quarter, 32-byte swizzle: the K-major MMA
// layout).  Persistent CTAs, one per SM, walk the tiles: lane 0 of warp 0
// loads, lane 0 of warp 1 issues the 28 UMMAs of each quarter and hands each
// finished chunk to warps 2-17, which drain TMEM (lane quarter w % 4, columns
// [16 h + 64 g, 16 h + 64 g + 16), h = (w - 2) / 4, g < N / 64) into registers, release it, and write C
// (and, for the solve, the digit planes of C's new columns of F) while the
// next tile's products run.  Every wait is bounded (about one second); on a
// timeout the CTA sets bit 2 of flags, waits (bounded) for its own copies and
// MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "factor.cuh"
#include "oz_digits.cuh"
#include "ozgemm.cuh"
#include "tc_ptx.cuh"

namespace kevd {

namespace {

constexpr int kQ = 16;
constexpr int kChunk = 16;
constexpr int kDrainWarps = 16;
constexpr int kThreads = (2 + kDrainWarps) * 32;
constexpr int kM = 128;
constexpr uint32_t kPlaneA = kM * 32;                    // one plane of a quarter: 128 rows x 32 bytes
constexpr uint32_t kCols = 512;                          // TMEM: 7 accumulators x 64 or 3 x 128 columns

// B rows per tile for a digit count: 64 for seven digits (seven accumulators), 128
// for three (three accumulators of 128 columns).
__host__ __device__ constexpr int oz_tile_n(int D) { return D == 3 ? 128 : 64; }

// Per digit count D (7: FP64 operands, 3: FP32 operands): the tile's B rows, the
// stage of one quarter (D planes of A and of B) and the ring depth.
template <int D>
struct OzCfg {
    static constexpr int kN = oz_tile_n(D);
    static constexpr uint32_t kPlaneB = kN * 32;
    static constexpr int kStages = D >= 6 ? 5 : 8;
    static constexpr uint32_t kStageA = D * kPlaneA;
    static constexpr uint32_t kStage = kStageA + D * kPlaneB;
    static constexpr size_t kSmem = (size_t)kStages * kStage + 1024;
    static_assert(kSmem <= 227 * 1024, "shared memory");
    static_assert(D * kN <= (int)kCols, "TMEM");
};

// TMEM accumulator of the pair (s, lv - s) of level lv (acc_of for seven digits).
template <int D>
__device__ __forceinline__ constexpr int accD(int lv, int s) {
    return D == 7 ? acc_of(lv, s) : lv;
}

// 2^sc (T + M 2^24) for the INT64 and FP32 sums of one entry with a single FP64
// operation (FP64 is the slow pipe): T and M become doubles by bit assembly
// (exact: |T| < 2^53 for contractions below 2^17 columns, M normal or
// negligible), one FMA, and the scale by an exponent add when it stays normal.
__device__ __forceinline__ double oz_combine(long long T, float M, int sc) {
    double td = 0.0;
    if (T != 0) {
        const unsigned long long u = T < 0 ? (unsigned long long)(-T) : (unsigned long long)T;
        const int msb = 63 - __clzll(u);
        if (msb <= 52) {
            td = __longlong_as_double((long long)(((unsigned long long)(T < 0) << 63) |
                                                  ((unsigned long long)(msb + 1023) << 52) |
                                                  ((u << (52 - msb)) & 0xFFFFFFFFFFFFFull)));
        } else {
            td = (double)T;
        }
    }
    double md = 0.0;
    const uint32_t mb = __float_as_uint(M);
    const uint32_t me = (mb >> 23) & 0xFF;
    if (me != 0 && me != 0xFF)
        md = __longlong_as_double((long long)(((unsigned long long)(mb >> 31) << 63) |
                                              ((unsigned long long)(me - 127 + 1023) << 52) |
                                              ((unsigned long long)(mb & 0x7FFFFF) << 29)));
    const double t = fma(md, 0x1p24, td);
    const long long b = __double_as_longlong(t);
    const int be = (int)((b >> 52) & 0x7FF);
    if ((b & 0x7FFFFFFFFFFFFFFFll) == 0) return t;                  // zero (integer test: no FP64 compare)
    if (be + sc >= 1 && be + sc <= 2046) return __longlong_as_double(b + ((long long)sc << 52));
    return ldexp(t, sc);
}

// D digits (levels 0 .. D - 1 of the pairs s + t <= D - 1; D = 3 or 7).  rowdiv:
// C(i, :) is divided by rowdiv[i] (one reciprocal per row), when not NULL.
template <int D>
__global__ void __launch_bounds__(kThreads, 1)
    k_ozmm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const int* __restrict__ ea,
           int ea_const, const int* __restrict__ eb, int eb_const, int64_t M, int n, int K,
           const FactorState* __restrict__ st, double* __restrict__ Cout, int64_t ldc, int64_t c_koff,
           uint16_t* __restrict__ pout, int64_t pout_ld, int64_t pout_plane, const double* __restrict__ rowdiv,
           int* __restrict__ flags) {
    constexpr int kN = OzCfg<D>::kN;
    constexpr int kNH = kN / 64;                               // 16-column groups per drain warp
    constexpr uint32_t kPlaneB = OzCfg<D>::kPlaneB;
    constexpr uint32_t kIdesc = idesc_bf16(kM, kN);
    constexpr int kStages = OzCfg<D>::kStages;
    constexpr uint32_t kStageA = OzCfg<D>::kStageA;
    constexpr uint32_t kStage = OzCfg<D>::kStage;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * kStages + 2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;

    int ncols = n, pk = 0;
    if (st) {   // engine products: skipped rounds write nothing
        if (st->done || st->m == 0) return;
        if (K == -1) K = st->k;                                  // contraction over the current rank
        if (K == -2) K = st->m;                                  // ... over this round's pivots
        if (K == -3) K = st->kp;                                 // ... over F's padded planes
        if (c_koff) {                                            // output at columns k .. k + m - 1
            Cout += (int64_t)st->k * c_koff;
            pk = st->kp;
            ncols = min(n, st->m);
        }
    }
    // tiles: 128-row block rb, kN-column block jt, t = rb nj + jt (the j tiles of a row
    // block are neighbours, so they read A's planes at about the same time); CTA b
    // takes t = b, b + gridDim.x, ... and keeps the TMA ring and the MMAs running
    // across its tiles: a tile's epilogue overlaps the next tile's products
    const int nj = (n + kN - 1) / kN;
    const int64_t ntile = (M + kM - 1) / kM * nj;
    const int nq = (K + kQ - 1) / kQ;
    const int nchunk = (nq + kChunk - 1) / kChunk;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto full = [&](int64_t g) { return bar0 + 8u * (uint32_t)(g % kStages); };
    auto empty = [&](int64_t g) { return bar0 + 8u * (uint32_t)(kStages + g % kStages); };
    const uint32_t acc_full = bar0 + 8u * (2 * kStages);
    const uint32_t acc_empty = bar0 + 8u * (2 * kStages + 1);

    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            mbar_init(full(q), 1);
            mbar_init(empty(q), 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, kDrainWarps);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (wid == 0) {
        // ---- TMA producer: quarter g = (tile iteration) nq + q ----
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            int64_t g = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
                const int i0 = (int)(t / nj) * kM, j0 = (int)(t % nj) * kN;
                for (int q = 0; q < nq; ++q, ++g) {
                    if (g >= kStages && !mbar_wait_or_fail(empty(g), (uint32_t)(g / kStages - 1) & 1, &s_fail)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = base + (uint32_t)(g % kStages) * kStage;
                    mbar_expect_tx(full(g), kStage);
                    tma_load_3d(dst, &tmA, q * kQ, i0, 0, full(g));
                    tma_load_3d(dst + kStageA, &tmB, q * kQ, j0, 0, full(g));
                }
            }
            if (!ok) {
                s_fail = 1;
                atomicOr(flags, 4);
            }
            for (int64_t j = g > kStages ? g - kStages : 0; j < g; ++j) mbar_wait(full(j), (uint32_t)(j / kStages) & 1);
        }
    } else if (wid == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int64_t g = 0, c = 0, last = -1;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
                for (int q = 0; q < nq; ++q, ++g) {
                    const bool first = (q % kChunk) == 0;
                    if (first && c > 0 && !mbar_wait_or_fail(acc_empty, (uint32_t)(c - 1) & 1, &s_fail)) {
                        ok = false;
                        break;
                    }
                    if (!mbar_wait_or_fail(full(g), (uint32_t)(g / kStages) & 1, &s_fail)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + (uint32_t)(g % kStages) * kStage, sb = sa + kStageA;
#pragma unroll
                    for (int lv = 0; lv < D; ++lv) {
#pragma unroll
                        for (int s = 0; s <= lv; ++s) {
                            const bool lead = lv < 4 ? s == 0 : lv == 4 ? (s == 0 || s == 3) : (lv == 5 && s == 0);
                            umma_bf16(tmem + (uint32_t)kN * accD<D>(lv, s), sw32_desc(sa + s * kPlaneA),
                                      sw32_desc(sb + (lv - s) * kPlaneB), kIdesc, (first && lead) ? 0u : 1u);
                        }
                    }
                    umma_commit(empty(g));
                    last = g;
                    if ((q % kChunk) == kChunk - 1 || q == nq - 1) {
                        umma_commit(acc_full);
                        ++c;
                    }
                }
            }
            if (!ok) {
                s_fail = 1;
                atomicOr(flags, 4);
            }
            if (last >= 0) mbar_wait(empty(last), (uint32_t)(last / kStages) & 1);
        }
    } else {
        // ---- drain and epilogue: TMEM lane quarter wid % 4, columns [16 h + 64 g, + 16) ----
        const int wq = wid & 3, h = (wid - 2) >> 2;
        const int m = 32 * wq + lane;
        const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
        const int pcols = (ncols + kQ - 1) / kQ * kQ;   // new columns' planes: zeros past ncols up to 16
        int64_t c = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            const int64_t i0 = (t / nj) * kM;
            const int j0 = (int)(t % nj) * kN;
            long long Tacc[16 * kNH];
            float Macc[16 * kNH];
#pragma unroll
            for (int e = 0; e < 16 * kNH; ++e) {
                Tacc[e] = 0;
                Macc[e] = 0.f;
            }
            for (int ch = 0; ch < nchunk; ++ch, ++c) {
                if (!mbar_wait_sleep(acc_full, (uint32_t)c & 1, &s_fail, 64)) {
                    ok = false;
                    break;
                }
                __syncwarp();
                tc_fence_after();
#pragma unroll
                for (int half = 0; half < kNH; ++half) {
                    const uint32_t col = (uint32_t)(16 * h + 64 * half);
#pragma unroll
                    for (int gl = 0; gl < (D < 4 ? D : 4); ++gl) {
                        uint32_t r[16];
                        tmem_ld16_async(tmem + lane_off + (uint32_t)(kN * gl) + col, r);
                        tmem_wait_ld16(r);
                        const float up = __int_as_float((127 + 8 * gl) << 23);
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            Tacc[16 * half + e] += (long long)__float2int_rn(__uint_as_float(r[e]) * up) << (24 - 8 * gl);
                    }
                    // level 4, one exact half at a time (units 2^-32): whole 2^-24 units to Tacc,
                    // the rest to Macc (the two halves' floors and residues add up to the sum's)
                    uint32_t r[16];
                    #pragma unroll
                    for (int hf = 4; hf <= (D > 4 ? 5 : 3); ++hf) {
                        tmem_ld16_async(tmem + lane_off + (uint32_t)(kN * hf) + col, r);
                        tmem_wait_ld16(r);
                    #pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int i4 = __float2int_rn(__uint_as_float(r[e]) * 0x1p32f);
                            Tacc[16 * half + e] += (long long)(i4 >> 8);
                            Macc[16 * half + e] += (float)(i4 & 255) * 0x1p-32f;
                        }
                    }
                    if (D > 5) {
                        tmem_ld16_async(tmem + lane_off + (uint32_t)(kN * 6) + col, r);
                        tmem_wait_ld16(r);
#pragma unroll
                        for (int e = 0; e < 16; ++e) Macc[16 * half + e] += __uint_as_float(r[e]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);          // TMEM free for the next chunk or tile
            }
            if (!ok) break;
            const int64_t gi = i0 + m;
            if (gi < M && D == kDigits && pout) {
                // the solve: C and the seven planes of its 16 columns (exponent 1), each
                // plane's 32 bytes of the row as two 16-byte stores
                const int ei = ea ? ea[gi] : ea_const;
                long long Tq[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int gj = j0 + 16 * h + e;
                    double v = 0.0;
                    if (gj < ncols) {
                        const int ej = eb ? eb[gj] : eb_const;
                        if (ei > -900 && ej > -900) v = oz_combine(Tacc[e], Macc[e], ei + ej - 36);
                        Cout[gi + (int64_t)gj * ldc] = v;
                    }
                    Tq[e] = oz_T_f64<kDigits>(v, 1);
                }
                if (j0 + 16 * h < pcols) {
                    uint16_t* dst = pout + gi * pout_ld + pk + j0 + 16 * h;
#pragma unroll
                    for (int s = 0; s < kDigits; ++s) {
                        uint32_t wv[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) wv[j] = oz_word<kDigits>(Tq[2 * j], Tq[2 * j + 1], s);
                        uint4* q4 = reinterpret_cast<uint4*>(dst + (size_t)s * pout_plane);
                        q4[0] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                        q4[1] = make_uint4(wv[4], wv[5], wv[6], wv[7]);
                    }
                }
            } else if (gi < M) {
                const int ei = ea ? ea[gi] : ea_const;
                const double dinv = rowdiv ? 1.0 / rowdiv[gi] : 1.0;
#pragma unroll
                for (int e = 0; e < 16 * kNH; ++e) {
                    const int gj = j0 + 64 * (e / 16) + 16 * h + e % 16;
                    if (gj < ncols) {
                        const int ej = eb ? eb[gj] : eb_const;
                        double v = 0.0;
                        if (ei > -900 && ej > -900) v = oz_combine(Tacc[e], Macc[e], ei + ej - 36);
                        Cout[gi + (int64_t)gj * ldc] = rowdiv ? v * dinv : v;
                    }
                }
            }
        }
        if (!ok && lane == 0) {
            s_fail = 1;
            atomicOr(flags, 4);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

typedef CUresult (*EncodeFnMM)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFnMM encoder_mm() {
    static EncodeFnMM fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFnMM>(p);
    }
    return fn;
}

}  // namespace

bool ozmm_map(CUtensorMap* map, const uint16_t* planes, int64_t rows, int64_t ldk, int64_t plane, bool a_side,
              int digits) {
    EncodeFnMM enc = encoder_mm();
    if (!enc || !planes || (reinterpret_cast<uintptr_t>(planes) % 16) || ldk % 16 || plane % 8 || rows < 1 ||
        (digits != 3 && digits != kDigits))
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)ldk, (cuuint64_t)rows, (cuuint64_t)digits};
    const cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)plane * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kQ, (cuuint32_t)(a_side ? kM : oz_tile_n(digits)), (cuuint32_t)digits};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(planes), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int D>
static cudaError_t launch_ozmm_d(const CUtensorMap& ma, const CUtensorMap& mb, const int* ea, int ea_const,
                                 const int* eb, int eb_const, int64_t M, int n, int K, const FactorState* st,
                                 double* C, int64_t ldc, int64_t c_koff, uint16_t* pout, int64_t pout_ld,
                                 int64_t pout_plane, const double* rowdiv, int* flags, int sms, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_ozmm<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)OzCfg<D>::kSmem);
    if (e != cudaSuccess) return e;
    const int64_t ntile = (M + kM - 1) / kM * ((n + OzCfg<D>::kN - 1) / OzCfg<D>::kN);
    const dim3 grid((unsigned)std::min<int64_t>(ntile, sms));   // persistent: one CTA per SM
    k_ozmm<D><<<grid, kThreads, OzCfg<D>::kSmem, s>>>(ma, mb, ea, ea_const, eb, eb_const, M, n, K, st, C, ldc, c_koff,
                                                      pout, pout_ld, pout_plane, rowdiv, flags);
    return cudaGetLastError();
}

cudaError_t launch_ozmm(const CUtensorMap& ma, const CUtensorMap& mb, const int* ea, int ea_const, const int* eb,
                        int eb_const, int64_t M, int n, int K, const FactorState* st, double* C, int64_t ldc,
                        int64_t c_koff, uint16_t* pout, int64_t pout_ld, int64_t pout_plane, int* flags,
                        cudaStream_t s, int digits, const double* rowdiv) {
    if (M < 1 || n < 1 || M >= ((int64_t)1 << 31) || (digits != 3 && digits != kDigits)) return cudaErrorInvalidValue;
    if (pout && (digits != kDigits || (reinterpret_cast<uintptr_t>(pout) % 16) || pout_ld % 16 || pout_plane % 8))
        return cudaErrorInvalidValue;
    static int nsm[64] = {};
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int sms = dev >= 0 && dev < 64 ? nsm[dev] : 0;
    if (sms == 0) {
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) nsm[dev] = sms;
    }
    if (digits == 3)
        return launch_ozmm_d<3>(ma, mb, ea, ea_const, eb, eb_const, M, n, K, st, C, ldc, c_koff, pout, pout_ld,
                                pout_plane, rowdiv, flags, sms, s);
    return launch_ozmm_d<kDigits>(ma, mb, ea, ea_const, eb, eb_const, M, n, K, st, C, ldc, c_koff, pout, pout_ld,
                                  pout_plane, rowdiv, flags, sms, s);
}

}  // namespace kevd
