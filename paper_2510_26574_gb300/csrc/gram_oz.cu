// Weighted Gram matrices of an FP64 factor on the tensor cores at FP64
// accuracy: A = F^T diag(wa) F and C = F^T diag(wc) F (Section 2.2), by an
// error-free slicing of the operands in the manner of Ozaki, Ogita, Oishi and
// Rump (2012), with BF16 slice products summed exactly in TMEM.
//
// Slicing.  Every operand column c (over all rows) has an exponent E_c with
// max_i |x_ic| < 2^E_c.  T = round(x 2^(46 - E_c)) is an integer below 2^46,
// written in six balanced base-256 digits d_0 .. d_5 (d_s in [-128, 127]), so
// x = 2^(E_c - 6) sum_s d_s 2^(-8 s) up to 2^(E_c - 47).  Digit plane s holds
// p_s = d_s 2^(-8 s), an exact BF16 value.
//
// Products.  The Gram entry is 2^(E_u + E_v - 12) sum_(s,t) sum_i p_s p_t; the
// pairs with s + t <= 5 are kept (21 MMAs per 16 rows), the rest lie below
// 2^-48 of the largest product.  Level g = s + t has g + 1 pairs whose
// products are integer multiples of 2^(-8 g) below 2^14 in magnitude, so over
// 256 rows the level-g sum is an integer multiple of 2^(-8 g) below 2^24 for
// g <= 3: exact in an FP32 TMEM accumulator, whatever its rounding.  Levels 0-3
// have one accumulator each, level 4 two (pairs s <= 2 and s >= 3, each below
// 2^24 units of 2^-32: exact too) and level 5 a seventh.  One accumulator for
// levels 4 and 5 would not do: the tensor core truncates each addend to the
// accumulator's ulp, a bias that reaches ~2^-48 of the total over a chunk.
//
// Accumulation.  After every 256-row chunk the drain turns levels 0-4 into one
// integer I_0 2^24 + I_1 2^16 + I_2 2^8 + I_3 + floor(I_4 / 2^8) (I_g = L_g
// 2^(8 g), exact FP32-to-integer conversions) added to an INT64 running sum,
// and the rest of level 4 (I_4 mod 2^8, times 2^-32) and level 5 into an FP32
// running sum.  No FP64 arithmetic runs per chunk; the column
// scales 2^(E_u + E_v - 12) and the conversion to FP64 are applied once at the
// end, and the row splits are added in FP64 afterwards.
//
// Per CTA: one tile of M = 128 columns of the I block (U = F(:, I), unweighted)
// by N = 64 columns of the J block (V = w F(:, J), w = wa or wc by
// blockIdx.z), over one range of rows.  Sixteen warps; rows move in 16-row
// quarter stages (one K step of the MMA):
//   * lane 0 of warp 0 keeps a three-slot ring of raw FP64 quarters filled:
//     TMA loads (cp.async.bulk.tensor, 16 rows x 64 columns: two for the I
//     block, one for the J block; zero fill past N and past rank) and a bulk
//     copy of the weights, issued for quarter q + 3 once every warp has read q;
//   * all warps cut each raw quarter into the six digit planes of U and V in
//     the 128-byte swizzled K-major layout of a 64-row slice stage, whose four
//     quarters alternate with the MMAs (the MMAs of quarter q run while the
//     slicers fill q + 1);
//   * lane 0 of warp 0, after waiting for all warps on the quarter's mbarrier,
//     issues its 21 UMMAs, committed back to the slicers and, at the end of a
//     256-row chunk, to the drain;
//   * all warps drain after each chunk (warp w reads TMEM lane quarter w % 4,
//     tile columns [16 (w / 4), 16 (w / 4) + 16)).
// Every wait is bounded (about one second); on a timeout the CTA sets bit 2 of
// flags, waits (bounded) for its own copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "gram_tc.cuh"
#include "tc_ptx.cuh"

namespace kevd {

constexpr int kOzQ = 16;          // rows per quarter stage (one MMA K step)
constexpr int kOzSlots = 3;       // raw quarters in flight
constexpr int kOzChunk = 16;      // quarters per exact chunk: 256 rows
constexpr int kOzDigits = 6;
constexpr int kOzWarps = 16;
constexpr int kOzThreads = kOzWarps * 32;
constexpr int kOzM = 128, kOzN = 64;
constexpr uint32_t kOzRawI = kOzM * kOzQ * 8;           // raw FP64 I block, [column][row]: 16 KB
constexpr uint32_t kOzRawJ = kOzN * kOzQ * 8;           // 8 KB
constexpr uint32_t kOzRawW = kOzQ * 8;                  // 128 B of weights
constexpr uint32_t kOzRaw = kOzRawI + kOzRawJ + kOzRawW;
constexpr uint32_t kOzPlaneU = kOzM * 128;              // one digit plane: 128 rows x 64 BF16 (16 KB)
constexpr uint32_t kOzPlaneV = kOzN * 128;              // 8 KB
constexpr uint32_t kOzSlice = kOzDigits * (kOzPlaneU + kOzPlaneV);
constexpr uint32_t kOzCols = 512;                       // TMEM: 7 accumulators x 64 columns (allocation: 512)
constexpr size_t kOzSmem = (size_t)kOzSlice + kOzSlots * (size_t)kOzRaw + 1024;

// Tile t -> (I, J) over I-blocks of 128 columns and J-blocks of 64 columns
// with J >= 2 I (the tiles holding some entry a <= c).
__device__ __forceinline__ void oz_tile_decode(int t, int nbi, int nbj, int& I, int& J) {
    I = 0;
    int len = nbj;
    while (t >= len && I + 1 < nbi) {
        t -= len;
        ++I;
        len = nbj - 2 * I;
    }
    J = 2 * I + t;
}

int oz_ntiles(int rank) {
    const int nbi = (rank + kOzM - 1) / kOzM, nbj = (rank + kOzN - 1) / kOzN;
    int n = 0;
    for (int I = 0; I < nbi; ++I) n += nbj - 2 * I;
    return n;
}

// The six digit planes of 2 consecutive values of one column: p_s = d_s 2^(-8 s)
// as BF16, packed two rows per 32-bit word (plane s in w[s]).  sh0 = 1029 + E, so
// that T = round(x 2^(46 - E)), |T| < 2^46.  The balanced digits are the bytes of
// T + 0x808080808080 minus 128 (T + C lies in [0, 2^48), and T = sum (b - 128)
// 256^j exactly); BF16 of d 2^(-8 s) comes from the magic M_s = 1.5 * 2^(23 - 8 s),
// whose ulp is 2^(-8 s): float(bits(M_s) + d) - M_s = d 2^(-8 s), at most 8
// significant bits, so the upper half of the word is the exact BF16.
static __device__ __forceinline__ void oz_digits2(double x0, double x1, int sh0, uint32_t (&w)[kOzDigits]) {
    unsigned long long U[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const double x = u ? x1 : x0;
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        const int e = (int)((b >> 52) & 0x7FF);
        const int sh = sh0 - e;                                   // >= 7 since |x| < 2^E
        long long T = 0;
        if (e != 0 && e != 0x7FF && sh >= 1 && sh < 62) {
            const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
            T = (long long)(((m >> (sh - 1)) + 1) >> 1);          // round half up on |x| 2^(46 - E)
            T = T < 0x3FFFFFFFFFFFll ? T : 0x3FFFFFFFFFFFll;      // |x| rounding up to 2^E
            if ((long long)b < 0) T = -T;
        }
        U[u] = (unsigned long long)(T + 0x808080808080ll);
    }
#pragma unroll
    for (int s = 0; s < kOzDigits; ++s) {
        const int bi = kOzDigits - 1 - s;                         // plane 0 is the most significant byte
        const float Ms = 1.5f * __int_as_float((150 - 8 * s) << 23);
        const uint32_t mb = __float_as_uint(Ms) - 128u;
        const float f0 = __fsub_rn(__uint_as_float(mb + (uint32_t)((U[0] >> (8 * bi)) & 255u)), Ms);
        const float f1 = __fsub_rn(__uint_as_float(mb + (uint32_t)((U[1] >> (8 * bi)) & 255u)), Ms);
        w[s] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
    }
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_gram_oz(const __grid_constant__ CUtensorMap tmF, const double* __restrict__ wa, const double* __restrict__ wc,
              const int* __restrict__ Ecol, int rank, int64_t N, int nbi, int nbj, int64_t per,
              double* __restrict__ gpart, int ntiles, int* __restrict__ flags) {
    constexpr uint32_t kIdesc = idesc_bf16(kOzM, kOzN);
    extern __shared__ uint8_t smem_raw[];
    // raw_full[3], raw_empty[3], sl_full[4], sl_empty[4], acc_full
    __shared__ __align__(8) uint64_t bars[2 * kOzSlots + 9];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;

    int I, J;
    oz_tile_decode(blockIdx.x, nbi, nbj, I, J);
    const int gram = blockIdx.z;                                   // 0: A (wa), 1: C (wc)
    const double* w = gram ? wc : wa;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const int nq = i0 < i1 ? (int)((i1 - i0 + kOzQ - 1) / kOzQ) : 0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool issuer = tid == 0;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sl = base;                                      // digit planes (1024-aligned)
    const uint32_t rb0 = base + kOzSlice;                          // raw ring
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto raw_full = [&](int q) { return bar0 + 8u * (q % kOzSlots); };
    auto raw_empty = [&](int q) { return bar0 + 8u * (kOzSlots + q % kOzSlots); };
    auto sl_full = [&](int q) { return bar0 + 8u * (2 * kOzSlots + (q & 3)); };
    auto sl_empty = [&](int q) { return bar0 + 8u * (2 * kOzSlots + 4 + (q & 3)); };
    const uint32_t acc_full = bar0 + 8u * (2 * kOzSlots + 8);

    if (tid == 0) {
        for (int q = 0; q < kOzSlots; ++q) {
            mbar_init(raw_full(q), 1);
            mbar_init(raw_empty(q), kOzWarps);
        }
        for (int q = 0; q < 4; ++q) {
            mbar_init(sl_full(q), kOzWarps);
            mbar_init(sl_empty(q), 1);
        }
        mbar_init(acc_full, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kOzCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    auto load_quarter = [&](int q) {
        const int64_t row = i0 + (int64_t)q * kOzQ;
        const uint32_t dst = rb0 + (q % kOzSlots) * kOzRaw;
        mbar_expect_tx(raw_full(q), kOzRaw);
        tma_load_2d(dst, &tmF, (int)row, I * kOzM, raw_full(q));
        tma_load_2d(dst + kOzRawI / 2, &tmF, (int)row, I * kOzM + 64, raw_full(q));
        tma_load_2d(dst + kOzRawI, &tmF, (int)row, J * kOzN, raw_full(q));
        bulk_g2s(dst + kOzRawI + kOzRawJ, w + row, kOzRawW, raw_full(q));
    };
    int loaded = 0, last_q = -1;
    if (issuer) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmF)) : "memory");
        for (; loaded < kOzSlots && loaded < nq; ++loaded) load_quarter(loaded);
    }

    // slicing items, the same in every quarter: lane & 7 = 16-byte chunk of a raw
    // column (rows 2 k8, 2 k8 + 1 of the quarter); a warp takes columns
    // {b, b+2, b+4, b+6} (b = 8 (G / 2) + G % 2 for column group G), so that its
    // raw loads cover four whole 128-byte column rows and its 4-byte stores into
    // the swizzled planes meet 32 distinct banks.  Items: U columns from groups
    // wid and wid + 16, V columns from group wid.
    const int k8 = lane & 7, cq = lane >> 3;
    auto group_col = [](int G, int cqq) { return 8 * (G >> 1) + (G & 1) + 2 * cqq; };
    const int cu0 = group_col(wid, cq), cu1 = group_col(wid + 16, cq), cv = group_col(wid, cq);
    const int Eoff = gram ? 2 * rank : rank;
    auto shift_of = [&](int col, const int* E, bool ok) { return ok ? 1029 + E[col] : 4096; };
    const int shu0 = shift_of(I * kOzM + cu0, Ecol, I * kOzM + cu0 < rank);
    const int shu1 = shift_of(I * kOzM + cu1, Ecol, I * kOzM + cu1 < rank);
    const int shv = shift_of(J * kOzN + cv, Ecol + Eoff, J * kOzN + cv < rank);

    // drain: TMEM lane quarter wid % 4, tile columns [16 (wid / 4), + 16)
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
        const int qq = q & 3;                                      // quarter of the 64-row slice stage
        if (!mbar_wait_or_fail(raw_full(q), (uint32_t)(q / kOzSlots) & 1, &s_fail) ||
            (q >= 4 && !mbar_wait_or_fail(sl_empty(q), (uint32_t)((q >> 2) - 1) & 1, &s_fail))) {
            ok = false;
            break;
        }
        {
            const uint32_t rbase = rb0 + (q % kOzSlots) * kOzRaw;
            const int g = 2 * qq + (k8 >> 2);                      // 8-row group of the slice stage
            const uint32_t wo = 4 * (k8 & 3);                      // rows 2 k8, 2 k8 + 1 within the group
            double w0, w1;
            lds2d(rbase + kOzRawI + kOzRawJ + 16 * k8, w0, w1);
#pragma unroll 1
            for (int it = 0; it < 3; ++it) {
                const bool isv = it == 2;
                const int c = it == 0 ? cu0 : (it == 1 ? cu1 : cv);
                const int sh = it == 0 ? shu0 : (it == 1 ? shu1 : shv);
                double x0, x1;
                lds2d(rbase + (isv ? kOzRawI : 0u) + (uint32_t)c * (kOzQ * 8) + 16 * k8, x0, x1);
                if (isv) {
                    x0 = __dmul_rn(w0, x0);
                    x1 = __dmul_rn(w1, x1);
                }
                uint32_t wd[kOzDigits];
                oz_digits2(x0, x1, sh, wd);
                const uint32_t o = swz(c, g) + wo;
                const uint32_t pb = sl + (isv ? kOzDigits * kOzPlaneU : 0u);
                const uint32_t ps = isv ? kOzPlaneV : kOzPlaneU;
#pragma unroll
                for (int s = 0; s < kOzDigits; ++s) sts1(pb + s * ps + o, wd[s]);
            }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(sl_full(q));
            mbar_arrive(raw_empty(q));
        }
        const bool chunk_end = (q % kOzChunk) == kOzChunk - 1 || q == nq - 1;
        if (issuer) {
            if (!mbar_wait_or_fail(sl_full(q), (uint32_t)(q >> 2) & 1, &s_fail)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const bool first = (q % kOzChunk) == 0;
            const uint32_t off = 32u * qq;
            auto desc_u = [&](int s) { return sw128_desc(sl + s * kOzPlaneU + off); };
            auto desc_v = [&](int s) { return sw128_desc(sl + kOzDigits * kOzPlaneU + s * kOzPlaneV + off); };
            // accumulators (64 columns each): levels 0-3, level 4 as {s <= 2} and {s >= 3}, level 5
#pragma unroll
            for (int lv = 0; lv <= 5; ++lv) {
#pragma unroll
                for (int s = 0; s <= lv; ++s) {
                    const int a = lv < 4 ? lv : lv == 4 ? (s <= 2 ? 4 : 5) : 6;
                    const bool lead = s == 0 || (lv == 4 && s == 3);    // first MMA into this accumulator
                    umma_bf16(tmem + (uint32_t)kOzN * a, desc_u(s), desc_v(lv - s), kIdesc,
                              (first && lead) ? 0u : 1u);
                }
            }
            umma_commit(sl_empty(q));
            last_q = q;
            if (chunk_end) umma_commit(acc_full);
            if (loaded < nq) {
                if (!mbar_wait_or_fail(raw_empty(q), (uint32_t)(q / kOzSlots) & 1, &s_fail)) {
                    ok = false;
                    break;
                }
                load_quarter(loaded++);
            }
        }
        if (chunk_end) {
            __syncwarp();   // the issuer rejoins its warp: the TMEM loads are warp-collective
            if (!mbar_wait_or_fail(acc_full, (uint32_t)(q / kOzChunk) & 1, &s_fail)) {
                ok = false;
                break;
            }
            __syncwarp();
            tc_fence_after();
            // level g (0..3) adds L_g 2^(8 g) (an integer below 2^24, exact) at bit 24 - 8 g
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                uint32_t r[16];
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kOzN * g) + cb, r);
                tmem_wait_ld16(r);
                const float up = __int_as_float((127 + 8 * g) << 23);
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    Tacc[e] += (long long)__float2int_rn(__uint_as_float(r[e]) * up) << (24 - 8 * g);
            }
            {
                // level 4 (two exact halves, units 2^-32): whole 2^-24 units to Tacc, the rest to Macc
                uint32_t r[16], r2[16];
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kOzN * 4) + cb, r);
                tmem_wait_ld16(r);
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kOzN * 5) + cb, r2);
                tmem_wait_ld16(r2);
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int i4 = __float2int_rn(__uint_as_float(r[e]) * 0x1p32f) +
                                   __float2int_rn(__uint_as_float(r2[e]) * 0x1p32f);
                    Tacc[e] += (long long)(i4 >> 8);
                    Macc[e] += (float)(i4 & 255) * 0x1p-32f;
                }
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kOzN * 6) + cb, r);
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
        // entry (m, cb + e) = 2^(E_u + E_v - 12) (T 2^-24 + M); the FP64 partial of this split
        const int ri = I * kOzM + m;
        const int eu = ri < rank ? Ecol[ri] : 0;
        double* o = gpart + (((size_t)blockIdx.z * gridDim.y + blockIdx.y) * ntiles + blockIdx.x) * (kOzM * kOzN) +
                    (size_t)m * kOzN + cb;
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
            double v[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int rj = J * kOzN + cb + e + u;
                const int ev = rj < rank ? Ecol[Eoff + rj] : 0;
                v[u] = ldexp((double)Tacc[e + u] * 0x1p-24 + (double)Macc[e + u], eu + ev - 12);
            }
            *reinterpret_cast<double2*>(o + e) = make_double2(v[0], v[1]);
        }
    }
    if (issuer) {
        for (int j = loaded >= kOzSlots ? loaded - kOzSlots : 0; j < loaded; ++j)
            mbar_wait(raw_full(j), (uint32_t)(j / kOzSlots) & 1);
        if (last_q >= 0) mbar_wait(sl_empty(last_q), (uint32_t)(last_q >> 2) & 1);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzCols) : "memory");
}

// Column maxima of |F|, |wa F| and |wc F| for an FP64 factor, as the bits of
// non-negative doubles atomically maxed into cmax[0..3 rank) (zeroed before).
__global__ void __launch_bounds__(256) k_colmax3_f64(const double* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                                     int64_t per, const double* __restrict__ wa,
                                                     const double* __restrict__ wc,
                                                     unsigned long long* __restrict__ cmax) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= rank) return;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const double* col = F + (int64_t)c * ldf;
    double mu = 0.0, ma = 0.0, mc = 0.0;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
        const double x = col[i];
        mu = fmax(mu, fabs(x));
        ma = fmax(ma, fabs(__dmul_rn(wa[i], x)));
        if (wc) mc = fmax(mc, fabs(__dmul_rn(wc[i], x)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    if (lane == 0) {
        atomicMax(cmax + c, (unsigned long long)__double_as_longlong(mu));
        atomicMax(cmax + rank + c, (unsigned long long)__double_as_longlong(ma));
        atomicMax(cmax + 2 * rank + c, (unsigned long long)__double_as_longlong(mc));
    }
}

// E = the smallest integer with max < 2^E (frexp); zero or negligible
// (< 2^-900) columns get E = -900, which makes all their digits zero.
__global__ void k_colexp_f64(const unsigned long long* __restrict__ cmax, int n, int* __restrict__ E) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const double mx = __longlong_as_double((long long)cmax[c]);
    int e = -900;
    if (mx >= 0x1p-900) frexp(mx, &e);
    E[c] = e;
}

// Sum of the split partials in a fixed order; entry (a, c) of tile (I, J) is
// Gram entry (128 I + a, 64 J + c), written with its mirror when it lies in the
// upper triangle (each unordered pair has exactly one such owner).
__global__ void k_gram_oz_final(const double* __restrict__ gpart, int nsplit, int ntiles, int nbi, int nbj, int rank,
                                int ngram, double* __restrict__ A, double* __restrict__ C) {
    int I, J;
    oz_tile_decode(blockIdx.x, nbi, nbj, I, J);
    const int gram = blockIdx.y;
    if (gram >= ngram) return;
    double* G = gram ? C : A;
    for (int e = threadIdx.x; e < kOzM * kOzN; e += blockDim.x) {
        const int a = e / kOzN, c = e % kOzN;
        const int ra = I * kOzM + a, rc = J * kOzN + c;
        if (ra >= rank || rc >= rank || ra > rc) continue;
        double sum = 0.0;
        for (int q = 0; q < nsplit; ++q)
            sum += gpart[(((size_t)gram * nsplit + q) * ntiles + blockIdx.x) * (kOzM * kOzN) + e];
        G[(int64_t)rc * rank + ra] = sum;
        G[(int64_t)ra * rank + rc] = sum;
    }
}

bool gram_oz_eligible(const double* F, int64_t ldf, int64_t N, int rank) {
    if (const char* e = getenv("KEVD_GRAM")) {
        if (e[0] == 'f') return false;                          // KEVD_GRAM=fp64 / ffma: the FP64-pipe kernel
    }
    return rank >= 1 && N >= 1 && N < ((int64_t)1 << 31) && ldf % 2 == 0 &&
           (reinterpret_cast<uintptr_t>(F) % 16) == 0 && (uint64_t)ldf * 8 < ((uint64_t)1 << 40);
}

// Rows per split: a multiple of 64, at least 4,096 unless N is smaller, at most
// 2^22 (so that the INT64 sums cannot overflow), the split count chosen so that
// ntiles x nsplit x ngram CTAs fill whole waves of one CTA per SM.
int64_t gram_oz_per(int64_t N, int64_t nctas, int nsm, int* nsplit) {
    int64_t best_per = -1;
    double best_eff = -1.0;
    for (int64_t sp = 1; sp <= 64; ++sp) {
        const int64_t pr = ((N + sp - 1) / sp + 63) / 64 * 64;
        if (pr > ((int64_t)1 << 22)) continue;
        if (sp > 1 && pr < 4096) break;
        const int64_t ns = (N + pr - 1) / pr, blocks = nctas * ns;
        const double eff = (double)blocks / (double)(((blocks + nsm - 1) / nsm) * nsm);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best_per = pr;
        }
    }
    if (best_per < 0) best_per = (int64_t)1 << 22;
    *nsplit = (int)((N + best_per - 1) / best_per);
    return best_per;
}

size_t gram_oz_partial_doubles(int64_t N, int rank, int ngram, int nsm) {
    const int nt = oz_ntiles(rank);
    int ns = 1;
    gram_oz_per(N, (int64_t)nt * ngram, nsm, &ns);
    return (size_t)ngram * ns * nt * kOzM * kOzN;
}

typedef CUresult (*EncodeTiledFnOz)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t launch_gram_oz(const double* F, int64_t ldf, int64_t N, int rank, const double* wa, const double* wc,
                           unsigned long long* cmax, int* Ecol, double* gpart, int* flags, double* A, double* C,
                           int nsm, cudaStream_t s) {
    cudaError_t e;
    const int ngram = wc ? 2 : 1;
    if ((e = cudaMemsetAsync(cmax, 0, 3 * (size_t)rank * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    {
        const int ncs = (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 8192));
        const int64_t pr = ((N + ncs - 1) / ncs + 31) / 32 * 32;
        k_colmax3_f64<<<dim3((rank + 7) / 8, (unsigned)((N + pr - 1) / pr)), 256, 0, s>>>(F, ldf, N, rank, pr, wa, wc,
                                                                                           cmax);
        k_colexp_f64<<<(3 * rank + 255) / 256, 256, 0, s>>>(cmax, 3 * rank, Ecol);
    }
    static EncodeTiledFnOz enc = nullptr;
    if (!enc) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess)
            return cudaErrorNotSupported;
        enc = reinterpret_cast<EncodeTiledFnOz>(p);
    }
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rank};
    const cuuint64_t strides[1] = {(cuuint64_t)ldf * 8};
    const cuuint32_t box[2] = {(cuuint32_t)kOzQ, 64};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(F), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int nbi = (rank + kOzM - 1) / kOzM, nbj = (rank + kOzN - 1) / kOzN;
    const int nt = oz_ntiles(rank);
    int ns = 1;
    const int64_t per = gram_oz_per(N, (int64_t)nt * ngram, nsm, &ns);
    if ((e = cudaFuncSetAttribute(k_gram_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem)) !=
        cudaSuccess)
        return e;
    k_gram_oz<<<dim3((unsigned)nt, (unsigned)ns, (unsigned)ngram), kOzThreads, kOzSmem, s>>>(
        map, wa, wc, Ecol, rank, N, nbi, nbj, per, gpart, nt, flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_gram_oz_final<<<dim3((unsigned)nt, (unsigned)ngram), 256, 0, s>>>(gpart, ns, nt, nbi, nbj, rank, ngram, A, C);
    return cudaGetLastError();
}

}  // namespace kevd
