// FP64-accurate products C = A B^T on the tensor cores, contracting along the
// rows of A and B: C(i, j) = sum_c A(i, c) B(j, c), for the kernel-column
// engine of the FP64 path (Algorithm 2: X(:,:) X(S,:)^T and F(:, :k) F(S, :k)^T)
// and the lift U = D~^-1 F Y (Algorithm 1, last lines).
//
// Slicing (Ozaki, Ogita, Oishi and Rump, 2012, in an integer form, as in the
// FP64 Gram kernel but with seven digits): every row i of A has an exponent E_i
// with max_c |A(i, c)| < 2^E_i (from a bound amax_i supplied by the caller),
// likewise every row j of B.  T = x 2^(54 - E) holds all 53 bits of x (exact
// for |x| >= 2^(E - 1), rounded below that) in seven balanced base-256 digits,
// digit plane s holding d_s 2^(-8 s) as an exact BF16.  The 28 digit pairs
// with s + t <= 6 are formed (the rest lie below 2^-56 of the largest
// product: FP64 level, which the engine needs because its forward substitution
// amplifies product errors by the conditioning of L).  Levels 0-3 (g = s + t)
// and level 4 (in two halves) are summed exactly in FP32 TMEM accumulators
// over 256 columns of the contraction, levels 5-6 in a seventh; after each
// 256-column chunk the exact levels go into an INT64 running sum (units 2^-24,
// the sub-unit part of level 4 into the FP32 one) and levels 5-6 into an FP32
// one.
// C(i, j) = 2^(E_i + E_j - 12) (T 2^-24 + M), divided by rowdiv_i when given.
//
// Per CTA: M = 128 rows of A by N = 64 rows of B, the contraction in 16-column
// quarters.  A is read row-major (X: A(i, c) = X[i lda + c]) or column-major
// (F: A(i, c) = F[c lda + i]); B row-major.  Sixteen warps; lane 0 of warp 0
// keeps a five-slot TMA ring of raw FP64 quarters filled (four quarters ahead
// of the slicers, enough to cover the load latency) and issues the 28 UMMAs of
// each quarter once every warp has cut it into digit planes (a two-stage
// ring: the slicing of quarter q + 1 overlaps the MMAs of q); all warps drain
// after each chunk.  The contraction length may come from device
// memory (the engine's current rank), and the whole launch may be skipped by a
// device flag (a finished factorisation, or a round that accepted nothing).
// Every wait is bounded (about one second); on a timeout the CTA sets bit 2
// of flags, waits (bounded) for its own copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "factor.cuh"
#include "ozgemm.cuh"
#include "oz_digits.cuh"
#include "tc_ptx.cuh"

namespace kevd {

namespace {

constexpr int kQ = 16;            // contraction columns per quarter (one MMA K step)
constexpr int kSlots = 5;         // raw FP64 quarters in flight (TMA lead of four quarters)
constexpr int kStages = 2;        // digit-plane stages (slicing of q + 1 overlaps the MMAs of q)
constexpr int kChunk = 16;        // quarters per exact chunk: 256 columns
constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kM = 128, kN = 64;
constexpr uint32_t kRawA = kM * kQ * 8;                 // 16 KB
constexpr uint32_t kRawB = kN * kQ * 8;                 // 8 KB
constexpr uint32_t kRaw = kRawA + kRawB;
// Digit planes: block (s, stage) = one 32-byte K step of every row, the
// 14 blocks packed four to a 128-byte swizzled row (block b at plane b / 4,
// 32-byte slot b % 4), so the two stages of seven digits take four planes.
constexpr int kBlocks = kDigits * kStages;
constexpr int kPlanes = (kBlocks + 3) / 4;
constexpr uint32_t kPlaneA = kM * 128;                  // 16 KB
constexpr uint32_t kPlaneB = kN * 128;                  // 8 KB
constexpr uint32_t kSlice = kPlanes * (kPlaneA + kPlaneB);
constexpr uint32_t kCols = 512;    // TMEM: 7 accumulators x 64 columns
constexpr size_t kSmem = (size_t)kSlice + kSlots * (size_t)kRaw + 1024;
static_assert(kSmem <= 227 * 1024, "shared memory");

// Row i of the tile to the row group layout of a warp: rows {b, b+2, b+4, b+6}
// (b = 8 (G / 2) + G % 2) for 16-byte chunks of row-major raw data.
__device__ __forceinline__ int group_row(int G, int cq) { return 8 * (G >> 1) + (G & 1) + 2 * cq; }

template <bool ACOL>
__global__ void __launch_bounds__(kThreads, 1)
    k_ozgemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             const double* __restrict__ amax, const double* __restrict__ bmax, int64_t M, int n, int K,
             const FactorState* __restrict__ st, double* __restrict__ Cout, int64_t ldc, int64_t c_koff,
             const double* __restrict__ rowdiv, int* __restrict__ flags) {
    constexpr uint32_t kIdesc = idesc_bf16(kM, kN);
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * kSlots + 2 * kStages + 1];
    __shared__ int s_ej[kN];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;

    int ncols = n;
    if (st) {   // engine products: skipped rounds write nothing
        if (st->done || st->m == 0) return;
        if (K == -1) K = st->k;                                  // contraction over the current rank
        if (K == -2) K = st->m;                                  // ... or over this round's pivots
        if (c_koff) {                                            // output at columns k .. k + m - 1
            Cout += (int64_t)st->k * c_koff;
            ncols = min(n, st->m);
        }
    }
    const int64_t i0 = (int64_t)blockIdx.x * kM;
    const int j0 = blockIdx.y * kN;
    const int nq = (K + kQ - 1) / kQ;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool issuer = tid == 0;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sl = base;
    const uint32_t rb0 = base + kSlice;
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto raw_full = [&](int q) { return bar0 + 8u * (q % kSlots); };
    auto raw_empty = [&](int q) { return bar0 + 8u * (kSlots + q % kSlots); };
    auto sl_full = [&](int q) { return bar0 + 8u * (2 * kSlots + (q % kStages)); };
    auto sl_empty = [&](int q) { return bar0 + 8u * (2 * kSlots + kStages + (q % kStages)); };
    const uint32_t acc_full = bar0 + 8u * (2 * kSlots + 2 * kStages);
    // digit s of stage st: plane (2 s + st) / 4, 32-byte slot (2 s + st) % 4
    auto blk_plane = [](int s_, int st) { return (kStages * s_ + st) >> 2; };
    auto blk_slot = [](int s_, int st) { return (kStages * s_ + st) & 3; };

    if (tid < kN) s_ej[tid] = j0 + tid < n ? exp_of(bmax[j0 + tid]) : -900;
    if (tid == 0) {
        for (int q = 0; q < kSlots; ++q) {
            mbar_init(raw_full(q), 1);
            mbar_init(raw_empty(q), kWarps);
        }
        for (int q = 0; q < kStages; ++q) {
            mbar_init(sl_full(q), kWarps);
            mbar_init(sl_empty(q), 1);
        }
        mbar_init(acc_full, 1);
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

    auto load_quarter = [&](int q) {
        const int c0 = q * kQ;
        const uint32_t dst = rb0 + (q % kSlots) * kRaw;
        mbar_expect_tx(raw_full(q), kRaw);
        if (ACOL) tma_load_2d(dst, &tmA, (int)i0, c0, raw_full(q));     // [16 columns][128 rows]
        else tma_load_2d(dst, &tmA, c0, (int)i0, raw_full(q));          // [128 rows][16 columns]
        tma_load_2d(dst + kRawA, &tmB, c0, j0, raw_full(q));             // [64 rows][16 columns]
    };
    int loaded = 0, last_q = -1;
    if (issuer) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        for (; loaded < kSlots && loaded < nq; ++loaded) load_quarter(loaded);
    }

    // slicing items (fixed over quarters).  A row-major: rows group_row(wid), group_row(wid + 16)
    // of 16-byte chunk k8 (conflict-free loads and stores); A column-major: rows
    // 8 (G / 2) + (lane & 7) with k8 = 4 (G % 2) + lane / 8 for G = wid, wid + 16 (conflict-free
    // stores).  B: row group_row(wid, lane / 8), chunk lane & 7.
    const int k8b = lane & 7, cqb = lane >> 3;
    int ra[2], ka[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int G = wid + 16 * p;
        if (ACOL) {
            ra[p] = 8 * (G >> 1) + (lane & 7);
            ka[p] = 4 * (G & 1) + (lane >> 3);
        } else {
            ra[p] = group_row(G, cqb);
            ka[p] = k8b;
        }
    }
    const int rbv = group_row(wid, cqb);
    int sha[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int64_t gi = i0 + ra[p];
        const int ea = gi < M ? exp_of(amax[gi]) : -900;
        sha[p] = ea > -900 ? 1021 + ea : 4096;
    }
    const int ejb = exp_of(j0 + rbv < n ? bmax[j0 + rbv] : 0.0);
    const int shb = ejb > -900 ? 1021 + ejb : 4096;

    const int wq = wid & 3, cb = 16 * (wid >> 2);
    const int m = 32 * wq + lane;
    const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
    long long Tacc[16];
    float Macc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        Tacc[e] = 0;
        Macc[e] = 0.f;
    }
    bool ok = true;
    for (int q = 0; q < nq; ++q) {
        const int st = q % kStages;
        if (!mbar_wait_or_fail(raw_full(q), (uint32_t)(q / kSlots) & 1, &s_fail) ||
            (q >= kStages && !mbar_wait_or_fail(sl_empty(q), (uint32_t)(q / kStages - 1) & 1, &s_fail))) {
            ok = false;
            break;
        }
        {
            const uint32_t rbase = rb0 + (q % kSlots) * kRaw;
#pragma unroll 1
            for (int it = 0; it < 3; ++it) {
                const bool isb = it == 2;
                int row, k8, sh;
                double x0, x1;
                if (isb) {
                    row = rbv;
                    k8 = k8b;
                    sh = shb;
                    lds2d(rbase + kRawA + (uint32_t)row * (kQ * 8) + 16 * k8, x0, x1);
                } else {
                    row = it ? ra[1] : ra[0];
                    k8 = it ? ka[1] : ka[0];
                    sh = it ? sha[1] : sha[0];
                    if (ACOL) {
                        asm volatile("ld.shared.f64 %0, [%1];" : "=d"(x0) : "r"(rbase + (uint32_t)(2 * k8) * (kM * 8) + 8 * row));
                        asm volatile("ld.shared.f64 %0, [%1];" : "=d"(x1) : "r"(rbase + (uint32_t)(2 * k8 + 1) * (kM * 8) + 8 * row));
                    } else {
                        lds2d(rbase + (uint32_t)row * (kQ * 8) + 16 * k8, x0, x1);
                    }
                }
                uint32_t wd[kDigits];
                digits2(x0, x1, sh, wd);
                const uint32_t pb = sl + (isb ? kPlanes * kPlaneA : 0u);
                const uint32_t ps = isb ? kPlaneB : kPlaneA;
#pragma unroll
                for (int s = 0; s < kDigits; ++s)
                    sts1(pb + blk_plane(s, st) * ps + swz(row, 2 * blk_slot(s, st) + (k8 >> 2)) + 4 * (k8 & 3),
                         wd[s]);
            }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(sl_full(q));
            mbar_arrive(raw_empty(q));
        }
        const bool chunk_end = (q % kChunk) == kChunk - 1 || q == nq - 1;
        if (issuer) {
            if (!mbar_wait_or_fail(sl_full(q), (uint32_t)(q / kStages) & 1, &s_fail)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const bool first = (q % kChunk) == 0;
            const uint32_t slB = sl + kPlanes * kPlaneA;
#pragma unroll
            for (int lv = 0; lv < kDigits; ++lv) {
#pragma unroll
                for (int s = 0; s <= lv; ++s) {
                    const int t = lv - s;
                    const int a = acc_of(lv, s);
                    const bool lead = lv < 4 ? s == 0 : lv == 4 ? (s == 0 || s == 3) : (lv == 5 && s == 0);
                    umma_bf16(tmem + (uint32_t)kN * a,
                              sw128_desc(sl + blk_plane(s, st) * kPlaneA + 32u * blk_slot(s, st)),
                              sw128_desc(slB + blk_plane(t, st) * kPlaneB + 32u * blk_slot(t, st)), kIdesc,
                              (first && lead) ? 0u : 1u);
                }
            }
            umma_commit(sl_empty(q));
            last_q = q;
            if (chunk_end) umma_commit(acc_full);
            if (loaded < nq) {
                if (!mbar_wait_or_fail(raw_empty(q), (uint32_t)(q / kSlots) & 1, &s_fail)) {
                    ok = false;
                    break;
                }
                load_quarter(loaded++);
            }
        }
        if (chunk_end) {
            __syncwarp();
            if (!mbar_wait_or_fail(acc_full, (uint32_t)(q / kChunk) & 1, &s_fail)) {
                ok = false;
                break;
            }
            __syncwarp();
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                uint32_t r[16];
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kN * g) + cb, r);
                tmem_wait_ld16(r);
                const float up = __int_as_float((127 + 8 * g) << 23);
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    Tacc[e] += (long long)__float2int_rn(__uint_as_float(r[e]) * up) << (24 - 8 * g);
            }
            {
                // level 4 (two exact halves, units 2^-32): whole 2^-24 units to Tacc, the rest to Macc
                uint32_t r[16], r2[16];
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kN * 4) + cb, r);
                tmem_wait_ld16(r);
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kN * 5) + cb, r2);
                tmem_wait_ld16(r2);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int i4 = __float2int_rn(__uint_as_float(r[e]) * 0x1p32f) +
                                   __float2int_rn(__uint_as_float(r2[e]) * 0x1p32f);
                    Tacc[e] += (long long)(i4 >> 8);
                    Macc[e] += (float)(i4 & 255) * 0x1p-32f;
                }
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kN * 6) + cb, r);
                tmem_wait_ld16(r);
#pragma unroll
                for (int e = 0; e < 16; ++e) Macc[e] += __uint_as_float(r[e]);
            }
            tc_fence_before();
        }
    }
    if (!ok) {
        s_fail = 1;
        atomicOr(flags, 4);
    } else {
        // C = 2^(E_i + E_j - 36) (T + M 2^24): one FMA and one power-of-two scale per
        // entry (FP64 is the slow pipe here); the row divisor as one reciprocal per row
        const int64_t gi = i0 + m;
        if (gi < M) {
            const int ei = exp_of(amax[gi]);
            const double dinv = rowdiv ? 1.0 / rowdiv[gi] : 1.0;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int gj = j0 + cb + e;
                if (gj < ncols) {
                    const int ej = s_ej[cb + e];
                    double v = 0.0;
                    if (ei > -900 && ej > -900) {
                        v = fma((double)Macc[e], 0x1p24, (double)Tacc[e]);
                        const int sc = ei + ej - 36;
                        v = (sc >= -1022 && sc <= 1023) ? v * pow2(sc) : ldexp(v, sc);
                    }
                    Cout[gi + (int64_t)gj * ldc] = rowdiv ? v * dinv : v;
                }
            }
        }
    }
    if (issuer) {
        for (int j = loaded >= kSlots ? loaded - kSlots : 0; j < loaded; ++j)
            mbar_wait(raw_full(j), (uint32_t)(j / kSlots) & 1);
        if (last_q >= 0) mbar_wait(sl_empty(last_q), (uint32_t)(last_q / kStages) & 1);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                             const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                             CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

// 2D FP64 tensor map: inner dimension d0 (contiguous), outer d1 with row pitch ld.
bool map_f64(CUtensorMap* map, const double* base, uint64_t d0, uint64_t d1, uint64_t ld, uint32_t b0, uint32_t b1) {
    EncodeFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {d0, d1};
    const cuuint64_t strides[1] = {ld * 8};
    const cuuint32_t box[2] = {b0, b1};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool ozgemm_layout_ok(const double* p, int64_t ld) {
    return p && (reinterpret_cast<uintptr_t>(p) % 16) == 0 && ld % 2 == 0 && (uint64_t)ld * 8 < ((uint64_t)1 << 40);
}

cudaError_t launch_ozgemm(const double* A, int64_t lda, bool a_colmajor, int64_t M, const double* amax,
                          const double* B, int64_t ldb, int n, const double* bmax, int K, int Kmax,
                          const FactorState* st, double* C, int64_t ldc, const double* rowdiv, int* flags,
                          cudaStream_t s, int64_t c_koff) {
    if (M < 1 || n < 1 || Kmax < 1 || M >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    if (!ozgemm_layout_ok(A, lda) || !ozgemm_layout_ok(B, ldb)) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    const bool okA = a_colmajor ? map_f64(&ma, A, (uint64_t)M, (uint64_t)Kmax, (uint64_t)lda, kM, kQ)
                                : map_f64(&ma, A, (uint64_t)Kmax, (uint64_t)M, (uint64_t)lda, kQ, kM);
    if (!okA || !map_f64(&mb, B, (uint64_t)Kmax, (uint64_t)n, (uint64_t)ldb, kQ, kN)) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((M + kM - 1) / kM), (unsigned)((n + kN - 1) / kN));
    cudaError_t e;
    if (a_colmajor) {
        if ((e = cudaFuncSetAttribute(k_ozgemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) !=
            cudaSuccess)
            return e;
        k_ozgemm<true><<<grid, kThreads, kSmem, s>>>(ma, mb, amax, bmax, M, n, K, st, C, ldc, c_koff, rowdiv, flags);
    } else {
        if ((e = cudaFuncSetAttribute(k_ozgemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem)) !=
            cudaSuccess)
            return e;
        k_ozgemm<false><<<grid, kThreads, kSmem, s>>>(ma, mb, amax, bmax, M, n, K, st, C, ldc, c_koff, rowdiv, flags);
    }
    return cudaGetLastError();
}

}  // namespace kevd
