// Weighted Gram matrices of an FP64 factor on the tensor cores at FP64
// accuracy: A = F^T diag(wa) F and C = F^T diag(wc) F (Section 2.2), by an
// error-free slicing of the operands in the manner of Ozaki, Ogita, Oishi and
// Rump (2012), with BF16 slice products summed exactly in TMEM.
//
// Slicing.  Every operand column c (over all rows) has an exponent E_c with
// max_i |x_ic| < 2^E_c.  T = round(x 2^(46 - E_c)) is an integer below 2^46,
// written in six balanced base-256 digits d_0 .. d_5 (d_s in [-128, 127]), so
// x = 2^(E_c - 6) sum_s d_s 2^(-8 s) up to 2^(E_c - 47).  Digit plane s holds
// p_s = d_s 2^(-8 s), an exact BF16 value.  The operands are U = F (the I
// block of columns) and V = w F (the J block, w = wa or wc).
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
// running sum.  The column scales 2^(E_u + E_v - 12) and the conversion to
// FP64 are applied once per CTA, and the partials of row splits and slabs are
// added in FP64.
//
// Layout.  The rows are taken in slabs sized so that the digit planes of one
// slab stay within a fixed budget.  k_oz_planes cuts a slab once: for each of
// U, wa F (and wc F) six planes of rank_pad columns x S rows of BF16, a
// column's rows contiguous, so that a TMA box of 32 rows x 128 (or 64) columns
// x 6 planes with the 64-byte swizzle lands as six K-major MMA operands of two
// 16-row quarters (64-byte rows: half as many L2 requests per byte as 32-byte
// rows).  Every tile of the Gram reads those planes instead of cutting
// FP64 data itself (the cutting, not the MMAs, bounded the rate when each CTA
// sliced its own tiles).
//
// Per CTA of k_gram_oz: one tile of M = 128 columns of the I block by N = 64
// columns of the J block, for one Gram and one range of rows of the slab:
//   * lane 0 of warp 0 keeps a three-stage ring of 32-row stages filled (two
//     TMA loads per stage: 48 KB of U planes, 24 KB of V planes);
//   * lane 0 of warp 1 issues the 21 UMMAs of each quarter, frees a stage by a
//     commit, and at the end of each 256-row chunk commits to the drain and
//     waits for it before the next chunk overwrites the accumulators;
//   * warps 2-17 drain (TMEM lane quarter w % 4, tile columns [16 h, 16 h + 16)
//     with h = (w - 2) / 4) and finally add the tile's FP64 partial.
// Every wait is bounded (about one second); on a timeout the CTA sets bit 2 of
// flags, waits (bounded) for its own copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "gram_tc.cuh"
#include "tc_ptx.cuh"

namespace kevd {

constexpr int kOzQ = 16;          // rows per quarter (one MMA K step)
constexpr int kOzSQ = 2;          // quarters per stage (one 64-byte swizzled row of K)
constexpr int kOzStages = 3;      // stages in flight
constexpr int kOzChunk = 16;      // quarters per exact chunk: 256 rows
constexpr int kOzDigits = 6;
constexpr int kOzDrainWarps = 16;
constexpr int kOzThreads = (2 + kOzDrainWarps) * 32;
constexpr int kOzM = 128, kOzN = 64;
constexpr uint32_t kOzPlaneU = kOzM * 64;               // one digit plane of a stage: 128 columns x 64 bytes
constexpr uint32_t kOzPlaneV = kOzN * 64;               // 4 KB
constexpr uint32_t kOzStageU = kOzDigits * kOzPlaneU;   // 48 KB
constexpr uint32_t kOzStage = kOzStageU + kOzDigits * kOzPlaneV;   // 72 KB
constexpr uint32_t kOzCols = 512;                       // TMEM: 7 accumulators x 64 columns (allocation: 512)
constexpr size_t kOzSmem = (size_t)kOzStages * kOzStage + 1024;
constexpr size_t kOzPlaneBudget = (size_t)6 << 30;      // bytes of digit planes per slab
static_assert(kOzSmem <= 227 * 1024, "shared memory");

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

// Digit planes of the slab of rows [row0, row0 + rows) (rows a multiple of 16;
// zero past N and past rank): set 0 from F, set 1 from wa F, set 2 from wc F
// (when wc is given).  Plane (set, s) is rank_pad x S BF16 pairs, word
// ((set 6 + s) rank_pad + c) S / 2 + i / 2 holding rows i, i + 1 of column c.
// Block: 8 warps = 8 columns; a warp takes 64 rows per step (a lane two).
__global__ void __launch_bounds__(256) k_oz_planes(const double* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                                   int rank_pad, int64_t row0, int rows, int S,
                                                   const double* __restrict__ wa, const double* __restrict__ wc,
                                                   const int* __restrict__ Ecol, uint32_t* __restrict__ P) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= rank_pad) return;
    const bool on = c < rank;
    const size_t plane = (size_t)rank_pad * (S / 2);
    const int sets = wc ? 3 : 2;
    int sh[3];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
        const int e = (on && z < sets) ? Ecol[z * rank + c] : -900;
        sh[z] = e > -900 ? 1029 + e : 4096;
    }
    const double* col = F + (int64_t)c * ldf;
    for (int it = 0; it < 8; ++it) {
        const int il = blockIdx.y * 512 + it * 64 + 2 * lane;
        if (il >= rows) break;
        const int64_t i = row0 + il;
        double x0 = 0.0, x1 = 0.0;
        if (on && i + 1 < N) {
            const double2 v = *reinterpret_cast<const double2*>(col + i);
            x0 = v.x;
            x1 = v.y;
        } else if (on && i < N) {
            x0 = col[i];
        }
        const size_t at = (size_t)c * (S / 2) + (il >> 1);
#pragma unroll
        for (int z = 0; z < 3; ++z) {
            if (z >= sets) break;
            double y0 = x0, y1 = x1;
            if (z > 0) {
                const double* w = z == 1 ? wa : wc;
                y0 = i < N ? __dmul_rn(w[i], x0) : 0.0;
                y1 = i + 1 < N ? __dmul_rn(w[i + 1], x1) : 0.0;
            }
            uint32_t wd[kOzDigits];
            oz_digits2(y0, y1, sh[z], wd);
#pragma unroll
            for (int s = 0; s < kOzDigits; ++s) P[(size_t)(z * kOzDigits + s) * plane + at] = wd[s];
        }
    }
}

__device__ __forceinline__ int oz_acc(int lv, int s) { return lv < 4 ? lv : lv == 4 ? (s <= 2 ? 4 : 5) : 6; }

// One tile (I, J) of Gram blockIdx.z over rows [blockIdx.y per, + per) of the
// slab's planes (rows of the slab: `rows`); the FP64 result is stored into
// (accumulate = 0) or added to (accumulate = 1) its partial in gpart.
__global__ void __launch_bounds__(kOzThreads, 1)
    k_gram_oz(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmVA,
              const __grid_constant__ CUtensorMap tmVC, const int* __restrict__ Ecol, int rank, int rows, int nbi,
              int nbj, int per, double* __restrict__ gpart, int ntiles, int accumulate, int* __restrict__ flags) {
    constexpr uint32_t kIdesc = idesc_bf16(kOzM, kOzN);
    extern __shared__ uint8_t smem_raw[];
    // full[6], empty[6], acc_full, acc_empty
    __shared__ __align__(8) uint64_t bars[2 * kOzStages + 2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;

    int I, J;
    oz_tile_decode(blockIdx.x, nbi, nbj, I, J);
    const int gram = blockIdx.z;                                   // 0: A (wa), 1: C (wc)
    const int r0 = blockIdx.y * per, r1 = min(r0 + per, rows);
    const int nq = r0 < r1 ? (r1 - r0 + kOzQ - 1) / kOzQ : 0;
    const int nst = (nq + kOzSQ - 1) / kOzSQ;                     // stages (the last may hold one quarter)
    const int nchunk = (nq + kOzChunk - 1) / kOzChunk;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto full = [&](int q) { return bar0 + 8u * (q % kOzStages); };
    auto empty = [&](int q) { return bar0 + 8u * (kOzStages + q % kOzStages); };
    const uint32_t acc_full = bar0 + 8u * (2 * kOzStages);
    const uint32_t acc_empty = bar0 + 8u * (2 * kOzStages + 1);

    if (tid == 0) {
        for (int q = 0; q < kOzStages; ++q) {
            mbar_init(full(q), 1);
            mbar_init(empty(q), 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, kOzDrainWarps);
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
    const CUtensorMap* tmV = gram ? &tmVC : &tmVA;

    if (wid == 0) {
        // ---- TMA producer ----
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmU)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmV)) : "memory");
            int q = 0;                                             // stage index
            for (; q < nst; ++q) {
                if (q >= kOzStages &&
                    !mbar_wait_or_fail(empty(q), (uint32_t)(q / kOzStages - 1) & 1, &s_fail))
                    break;
                const uint32_t dst = base + (uint32_t)(q % kOzStages) * kOzStage;
                mbar_expect_tx(full(q), kOzStage);
                tma_load_3d(dst, &tmU, r0 + q * kOzSQ * kOzQ, I * kOzM, 0, full(q));
                tma_load_3d(dst + kOzStageU, tmV, r0 + q * kOzSQ * kOzQ, J * kOzN, 0, full(q));
            }
            if (q < nst) {
                s_fail = 1;
                atomicOr(flags, 4);
            }
            // before the CTA ends: the copies of the last stages have landed
            for (int j = std::max(0, q - kOzStages); j < q; ++j) mbar_wait(full(j), (uint32_t)(j / kOzStages) & 1);
        }
    } else if (wid == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int last = -1;
            bool ok = true;
            for (int g = 0; g < nst && ok; ++g) {                  // stage g: quarters 2 g, 2 g + 1
                if (!mbar_wait_or_fail(full(g), (uint32_t)(g / kOzStages) & 1, &s_fail)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t su = base + (uint32_t)(g % kOzStages) * kOzStage, sv = su + kOzStageU;
                for (int sub = 0; sub < kOzSQ; ++sub) {
                    const int q = g * kOzSQ + sub;
                    if (q >= nq) break;
                    const bool first = (q % kOzChunk) == 0;
                    if (first && q > 0 &&
                        !mbar_wait_or_fail(acc_empty, (uint32_t)(q / kOzChunk - 1) & 1, &s_fail)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t ko = 32u * sub;                    // second K step of the 64-byte row
#pragma unroll
                    for (int lv = 0; lv <= 5; ++lv) {
#pragma unroll
                        for (int s = 0; s <= lv; ++s) {
                            const bool lead = s == 0 || (lv == 4 && s == 3);    // first MMA into this accumulator
                            umma_bf16(tmem + (uint32_t)kOzN * oz_acc(lv, s), sw64_desc(su + s * kOzPlaneU + ko),
                                      sw64_desc(sv + (lv - s) * kOzPlaneV + ko), kIdesc, (first && lead) ? 0u : 1u);
                        }
                    }
                    if ((q % kOzChunk) == kOzChunk - 1 || q == nq - 1) umma_commit(acc_full);
                }
                umma_commit(empty(g));
                last = g;
            }
            if (!ok) {
                s_fail = 1;
                atomicOr(flags, 4);
            }
            if (last >= 0) mbar_wait(empty(last), (uint32_t)(last / kOzStages) & 1);   // own MMAs complete
        }
    } else {
        // ---- drain: TMEM lane quarter wid % 4, tile columns [16 h, 16 h + 16) ----
        const int wq = wid & 3, h = (wid - 2) >> 2;
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
        for (int c = 0; c < nchunk; ++c) {
            if (!mbar_wait_sleep(acc_full, (uint32_t)c & 1, &s_fail, 256)) {
                ok = false;
                break;
            }
            __syncwarp();
            tc_fence_after();
            {
                constexpr int half = 0;
                const uint32_t col = (uint32_t)(16 * h);
                // level g (0..3) adds L_g 2^(8 g) (an integer below 2^24, exact) at bit 24 - 8 g
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    uint32_t r[16];
                    tmem_ld16_async(tmem + lane_off + (uint32_t)(kOzN * g) + col, r);
                    tmem_wait_ld16(r);
                    const float up = __int_as_float((127 + 8 * g) << 23);
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        Tacc[16 * half + e] += (long long)__float2int_rn(__uint_as_float(r[e]) * up) << (24 - 8 * g);
                }
                // level 4, one exact half at a time (units 2^-32): whole 2^-24 units to Tacc,
                // the rest to Macc (the two halves' floors and residues add up to the sum's)
                uint32_t r[16];
                #pragma unroll
                for (int hf = 4; hf <= 5; ++hf) {
                    tmem_ld16_async(tmem + lane_off + (uint32_t)(kOzN * hf) + col, r);
                    tmem_wait_ld16(r);
                #pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int i4 = __float2int_rn(__uint_as_float(r[e]) * 0x1p32f);
                        Tacc[16 * half + e] += (long long)(i4 >> 8);
                        Macc[16 * half + e] += (float)(i4 & 255) * 0x1p-32f;
                    }
                }
                tmem_ld16_async(tmem + lane_off + (uint32_t)(kOzN * 6) + col, r);
                tmem_wait_ld16(r);
#pragma unroll
                for (int e = 0; e < 16; ++e) Macc[16 * half + e] += __uint_as_float(r[e]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
        }
        if (!ok) {
            if (lane == 0) {
                s_fail = 1;
                atomicOr(flags, 4);
            }
        } else if (nq > 0) {
            // entry (m, 32 h + e) = 2^(E_u + E_v - 36) (T + M 2^24), into this split's FP64 partial
            const int ri = I * kOzM + m;
            const int eu = ri < rank ? Ecol[ri] : -900;
            const int Eoff = gram ? 2 * rank : rank;
            double* o = gpart + (((size_t)gram * gridDim.y + blockIdx.y) * ntiles + blockIdx.x) * (kOzM * kOzN) +
                        (size_t)m * kOzN + 16 * h;
#pragma unroll
            for (int e = 0; e < 16; e += 2) {
                double v[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int rj = J * kOzN + 16 * h + e + u;
                    const int ev = rj < rank ? Ecol[Eoff + rj] : -900;
                    v[u] = 0.0;
                    if (eu > -900 && ev > -900)
                        v[u] = ldexp(fma((double)Macc[e + u], 0x1p24, (double)Tacc[e + u]), eu + ev - 36);
                }
                double2* dst = reinterpret_cast<double2*>(o + e);
                if (accumulate) {
                    const double2 old = *dst;
                    v[0] += old.x;
                    v[1] += old.y;
                }
                *dst = make_double2(v[0], v[1]);
            }
        } else if (!accumulate) {
            double* o = gpart + (((size_t)gram * gridDim.y + blockIdx.y) * ntiles + blockIdx.x) * (kOzM * kOzN) +
                        (size_t)m * kOzN + 16 * h;
            for (int e = 0; e < 16; ++e) o[e] = 0.0;
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzCols) : "memory");
}

// |x| as an FP32 value truncated toward zero (flushed to 0 below 2^-126), by bit
// manipulation on the integer pipe.
__device__ __forceinline__ float oz_abs_f32_rz(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    const int e = (int)(b >> 52) - 1023 + 127;
    if (e <= 0) return 0.f;
    if (e >= 255) return __uint_as_float(0x7F800000u);
    return __uint_as_float(((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
}

// |wa_i| and |wc_i| truncated to FP32, once per row (wc may be NULL).
__global__ void k_weights_rz(const double* __restrict__ wa, const double* __restrict__ wc, int64_t N,
                             float* __restrict__ wa_rz, float* __restrict__ wc_rz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    wa_rz[i] = oz_abs_f32_rz(wa[i]);
    if (wc) wc_rz[i] = oz_abs_f32_rz(wc[i]);
}

// Column bounds of |F|, |wa F| and |wc F| for an FP64 factor, as the bits of
// non-negative doubles atomically maxed into cmax[0..3 rank) (zeroed before).
// Only the exponent E with max < 2^E is needed, so the products are formed in
// FP32 from truncated copies (FP64 is the slow pipe; the weights' copies come
// from k_weights_rz) and the maxima raised by 2^-20: never below the true
// maximum, and the exponent one too high only when the maximum lies within 2^-20
// of a power of two.  |F| itself is exact.  Each warp reads its column in
// 256-row steps of four 16-byte vectors per lane when the column is 16-byte
// aligned (eight loads in flight per lane), then the ragged end row by row.
__global__ void __launch_bounds__(256) k_colmax3_f64(const double* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                                     int64_t per, const float* __restrict__ wa_rz,
                                                     const float* __restrict__ wc_rz,
                                                     unsigned long long* __restrict__ cmax) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= rank) return;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const double* col = F + (int64_t)c * ldf;
    unsigned long long mu = 0;
    float ma = 0.f, mc = 0.f;
    auto take = [&](double x, float a, float w) {
        mu = max(mu, (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull);
        const float xf = oz_abs_f32_rz(x);
        ma = fmaxf(ma, xf * a);
        mc = fmaxf(mc, xf * w);
    };
    int64_t i = i0;
    if ((reinterpret_cast<uintptr_t>(col + i0) & 15) == 0) {
        for (; i + 256 <= i1; i += 256) {
            double2 x[4];
            float2 a[4], w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t e = i + 64 * u + 2 * lane;
                x[u] = *reinterpret_cast<const double2*>(col + e);
                a[u] = *reinterpret_cast<const float2*>(wa_rz + e);
                w[u] = wc_rz ? *reinterpret_cast<const float2*>(wc_rz + e) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                take(x[u].x, a[u].x, w[u].x);
                take(x[u].y, a[u].y, w[u].y);
            }
        }
    }
    for (i += lane; i < i1; i += 32) take(col[i], wa_rz[i], wc_rz ? wc_rz[i] : 0.f);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mu = max(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    if (lane == 0) {
        const double up = 1.0 + 0x1p-20;
        atomicMax(cmax + c, mu);
        atomicMax(cmax + rank + c, (unsigned long long)__double_as_longlong((double)ma * up));
        atomicMax(cmax + 2 * rank + c, (unsigned long long)__double_as_longlong((double)mc * up));
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

static int oz_rank_pad(int rank) { return (rank + kOzM - 1) / kOzM * kOzM; }

// Rows per slab: a multiple of 256 (no more than N needs) with the planes of
// all sets within kOzPlaneBudget.
static int64_t oz_slab_rows(int64_t N, int rank, int ngram) {
    const size_t per_row = (size_t)(ngram + 1) * kOzDigits * oz_rank_pad(rank) * 2;
    int64_t S = (int64_t)(kOzPlaneBudget / per_row) / 256 * 256;
    S = std::max<int64_t>(S, 256);
    return std::min<int64_t>(S, (N + 255) / 256 * 256);
}

// Row splits per slab (the same in every slab): ntiles x ngram x nsplit CTAs
// filling whole waves of one CTA per SM, at least 4,096 rows per split.
static int oz_nsplit(int64_t S, int64_t nctas, int nsm) {
    int best = 1;
    double best_eff = -1.0;
    for (int sp = 1; sp <= 8; ++sp) {
        if (sp > 1 && S / sp < 4096) break;
        const int64_t blocks = nctas * sp;
        const double eff = (double)blocks / (double)(((blocks + nsm - 1) / nsm) * nsm);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = sp;
        }
    }
    return best;
}

size_t gram_oz_partial_doubles(int64_t N, int rank, int ngram, int nsm) {
    const int nt = oz_ntiles(rank);
    const int ns = oz_nsplit(oz_slab_rows(N, rank, ngram), (int64_t)nt * ngram, nsm);
    return (size_t)ngram * ns * nt * kOzM * kOzN;
}

size_t gram_oz_plane_bytes(int64_t N, int rank, int ngram) {
    return (size_t)(ngram + 1) * kOzDigits * oz_rank_pad(rank) * (size_t)oz_slab_rows(N, rank, ngram) * 2;
}

typedef CUresult (*EncodeTiledFnOz)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 3-D map over one set of planes (rows S, columns rank_pad, six digits), box
// 32 rows x `cols` columns x 6 digits with the 64-byte swizzle.
static bool oz_plane_map(EncodeTiledFnOz enc, CUtensorMap* map, uint16_t* base, int64_t S, int rank_pad, int cols) {
    const cuuint64_t dims[3] = {(cuuint64_t)S, (cuuint64_t)rank_pad, (cuuint64_t)kOzDigits};
    const cuuint64_t strides[2] = {(cuuint64_t)S * 2, (cuuint64_t)S * 2 * rank_pad};
    const cuuint32_t box[3] = {(cuuint32_t)(kOzSQ * kOzQ), (cuuint32_t)cols, (cuuint32_t)kOzDigits};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_gram_oz(const double* F, int64_t ldf, int64_t N, int rank, const double* wa, const double* wc,
                           float* wa_rz, float* wc_rz, unsigned long long* cmax, int* Ecol, double* gpart,
                           uint16_t* planes, int* flags, double* A, double* C, int nsm, cudaStream_t s) {
    cudaError_t e;
    const int ngram = wc ? 2 : 1;
    if ((e = cudaMemsetAsync(cmax, 0, 3 * (size_t)rank * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    {
        const int ncs = (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 8192));
        const int64_t pr = ((N + ncs - 1) / ncs + 255) / 256 * 256;
        k_weights_rz<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(wa, wc, N, wa_rz, wc ? wc_rz : nullptr);
        k_colmax3_f64<<<dim3((rank + 7) / 8, (unsigned)((N + pr - 1) / pr)), 256, 0, s>>>(
            F, ldf, N, rank, pr, wa_rz, wc ? wc_rz : nullptr, cmax);
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
    const int rank_pad = oz_rank_pad(rank);
    const int64_t S = oz_slab_rows(N, rank, ngram);
    const size_t set = (size_t)kOzDigits * rank_pad * S;          // BF16 elements per set
    CUtensorMap mu, mva, mvc;
    if (!oz_plane_map(enc, &mu, planes, S, rank_pad, kOzM) || !oz_plane_map(enc, &mva, planes + set, S, rank_pad, kOzN) ||
        !oz_plane_map(enc, &mvc, planes + (ngram == 2 ? 2 : 1) * set, S, rank_pad, kOzN))
        return cudaErrorInvalidValue;
    const int nbi = (rank + kOzM - 1) / kOzM, nbj = (rank + kOzN - 1) / kOzN;
    const int nt = oz_ntiles(rank);
    const int ns = oz_nsplit(S, (int64_t)nt * ngram, nsm);
    if ((e = cudaFuncSetAttribute(k_gram_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem)) !=
        cudaSuccess)
        return e;
    for (int64_t row0 = 0; row0 < N; row0 += S) {
        const int rows = (int)((std::min<int64_t>(S, N - row0) + kOzQ - 1) / kOzQ * kOzQ);
        k_oz_planes<<<dim3((unsigned)(rank_pad / 8), (unsigned)((rows + 511) / 512)), 256, 0, s>>>(
            F, ldf, N, rank, rank_pad, row0, rows, (int)S, wa, wc, Ecol, reinterpret_cast<uint32_t*>(planes));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int per = ((rows + ns - 1) / ns + kOzQ - 1) / kOzQ * kOzQ;
        k_gram_oz<<<dim3((unsigned)nt, (unsigned)ns, (unsigned)ngram), kOzThreads, kOzSmem, s>>>(
            mu, mva, mvc, Ecol, rank, rows, nbi, nbj, per, gpart, nt, row0 > 0 ? 1 : 0, flags);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_gram_oz_final<<<dim3((unsigned)nt, (unsigned)ngram), 256, 0, s>>>(gpart, ns, nt, nbi, nbj, rank, ngram, A, C);
    return cudaGetLastError();
}

}  // namespace kevd
