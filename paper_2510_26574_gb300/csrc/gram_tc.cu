// Weighted Gram matrices of an FP32 factor on the 5th-generation tensor cores
// (tcgen05 / TMEM): A = F^T diag(wa) F and C = F^T diag(wc) F, the two r x r
// products of the bistochastic normalisation (Section 2.2: B = D~^-1 F gives
// A = B^T B with wa = d~^-2; C = F^T Q~^-1 F with wc = 1/q~).
//
// Tensor-core FP32 accumulation does not round to nearest, and a Gram sums
// over all N rows, so plain split-BF16 products come out biased toward zero
// (~1e-5 relative, measured).  This kernel removes the bias by making the
// leading product exact:
//   * every operand column c (over all rows) gets a grid 2^(E_c - 7) with
//     max_i |x_ic| < 2^E_c; hi = x rounded to that grid is an integer in
//     [-128, 128] times 2^(E_c - 7), exactly a BF16 value, and
//     mid = bf16(x - hi) carries the next 8 bits;
//   * hi * hi products are integers below 2^14 in units of 2^(E_u + E_v - 14),
//     so their sums over up to 1,024 rows are integers below 2^24 in those
//     units: exact in the FP32 accumulator, whatever its rounding;
//   * the three other products (hi*mid, mid*hi, mid*mid) are ~2^-8 of the
//     total and go to a second accumulator, whose truncation error is ~2^-8
//     smaller again;
//   * every 1,024 rows both accumulators are added into FP32 running sums held
//     in registers (round to nearest), and the accumulators restart.
// The weights sit on the N side of the MMA, so one M = 128, N = 256 UMMA
// forms a 128 x 128 tile of both Grams: D[m][n] = sum_k F(k, I+m) V(k, n) with
// V = [wa F(:, J) | wc F(:, J)].
//
// Per CTA: one upper-triangular 128 x 128 tile pair (I, J) and one range of
// rows (a split; splits are added in FP64 afterwards).  Sixteen warps, each
// thread holding 64 FP32 running sums.  Rows move in 32-row half stages:
//   * lane 0 of warp 0 keeps a four-slot ring of raw half stages filled: TMA
//     loads (cp.async.bulk.tensor, 32 rows x 128 columns, zero fill past N and
//     past rank) of F(rows, I-block) and F(rows, J-block) and bulk copies of
//     the weights, issued for half stage q + 4 once every warp has read q;
//   * all warps slice each raw half stage into hi/mid BF16 in the 128-byte
//     swizzled K-major layout of a 64-row slice stage, whose two halves
//     alternate, so that slicing one half overlaps the MMAs of the other;
//   * lane 0 of warp 0, after waiting for all warps on the half's mbarrier,
//     issues its UMMAs (4 per 16 rows), committed back to the slicers and, at
//     the end of a 1,024-row chunk, to the drain;
//   * all warps drain the accumulators after each chunk (warp w reads TMEM
//     lane quarter w % 4, accumulator columns [64 (w / 4), 64 (w / 4) + 64)).
// Every wait is bounded (about one second); on a timeout the CTA sets bit 2
// of flags, waits (bounded) for its own copies and MMAs, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "gram_tc.cuh"
#include "tc_ptx.cuh"

namespace kevd {

constexpr int kGtHalf = 32;      // rows per half stage (the slice stage is 64 rows: one 128-byte K atom of BF16)
constexpr int kGtSlots = 4;      // raw half stages in flight
constexpr int kGtChunk = 32;     // half stages per exact accumulation chunk: 1,024 rows, sums <= 2^24
constexpr int kGtWarps = 16;
constexpr int kGtThreads = kGtWarps * 32;

template <bool TWO>
struct GtCfg {
    static constexpr int NV = TWO ? 256 : 128;                     // MMA N: [wa F_J | wc F_J] or [wa F_J]
    static constexpr uint32_t kRawF = 128 * kGtHalf * 4;           // raw FP32 block, [column][row]
    static constexpr uint32_t kRawW = kGtHalf * 4;
    static constexpr uint32_t kRaw = 2 * kRawF + 2 * kRawW;        // one raw half stage: F_I, F_J, wa, wc
    static constexpr uint32_t kU = 128 * 128;                      // one U slice: 128 x 64 BF16
    static constexpr uint32_t kV = NV * 128;                       // one V slice
    static constexpr uint32_t kSlice = 2 * kU + 2 * kV;            // U hi, U mid, V hi, V mid
    static constexpr uint32_t kCols = 2 * NV;                      // TMEM: level-0 and level-1 sums
    static constexpr size_t kSmem = kGtSlots * (size_t)kRaw + kSlice + 1024;
};

// hi = x rounded to the grid of the magic number M = 1.5 * 2^(E + 16) (whose
// ulp is 2^(E - 7)); mid = bf16(x - hi).  x - hi is exact in FP32.  Four
// values scaled by w: 8 bytes of each are stored at the shared addresses hi
// and mid.
static __device__ __forceinline__ void slice4(float4 x, float4 w, float M, uint32_t hi, uint32_t mid) {
    const float v[4] = {__fmul_rn(w.x, x.x), __fmul_rn(w.y, x.y), __fmul_rn(w.z, x.z), __fmul_rn(w.w, x.w)};
    uint32_t h[2], m[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float h0 = __fsub_rn(__fadd_rn(v[2 * e], M), M), h1 = __fsub_rn(__fadd_rn(v[2 * e + 1], M), M);
        // hi has at most 8 significant bits: the upper half of its FP32 word is
        // its exact BF16 encoding
        h[e] = __byte_perm(__float_as_uint(h0), __float_as_uint(h1), 0x7632);
        const __nv_bfloat162 mm = __floats2bfloat162_rn(__fsub_rn(v[2 * e], h0), __fsub_rn(v[2 * e + 1], h1));
        m[e] = *reinterpret_cast<const uint32_t*>(&mm);
    }
    sts2(hi, h[0], h[1]);
    sts2(mid, m[0], m[1]);
}

template <bool TWO>
__global__ void __launch_bounds__(kGtThreads, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmF, const float* __restrict__ wa, const float* __restrict__ wc,
              const float* __restrict__ mag, int rank, int64_t N, int nb, int64_t per, float* __restrict__ gpart,
              int ntri, int* __restrict__ flags) {
    using Cfg = GtCfg<TWO>;
    constexpr int NV = Cfg::NV;
    constexpr int CW = NV / 4;                                     // accumulator columns drained per thread
    constexpr uint32_t kIdesc = idesc_bf16(128, NV);
    extern __shared__ uint8_t smem_raw[];
    // raw_full[4], raw_empty[4], sl_full[2], sl_empty[2], acc_full
    __shared__ __align__(8) uint64_t bars[2 * kGtSlots + 5];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;

    int I, J;
    tri_decode(blockIdx.x, nb, I, J);
    const bool diag = I == J;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const int nq = i0 < i1 ? (int)((i1 - i0 + kGtHalf - 1) / kGtHalf) : 0;   // half stages
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool issuer = tid == 0;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sl = base + kGtSlots * Cfg::kRaw;               // slice stage (1024-aligned)
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto raw_full = [&](int q) { return bar0 + 8u * (q % kGtSlots); };
    auto raw_empty = [&](int q) { return bar0 + 8u * (kGtSlots + q % kGtSlots); };
    auto sl_full = [&](int h) { return bar0 + 8u * (2 * kGtSlots + h); };
    auto sl_empty = [&](int h) { return bar0 + 8u * (2 * kGtSlots + 2 + h); };
    const uint32_t acc_full = bar0 + 8u * (2 * kGtSlots + 4);

    if (tid == 0) {
        for (int q = 0; q < kGtSlots; ++q) {
            mbar_init(raw_full(q), 1);
            mbar_init(raw_empty(q), kGtWarps);
        }
        for (int h = 0; h < 2; ++h) {
            mbar_init(sl_full(h), kGtWarps);
            mbar_init(sl_empty(h), 1);
        }
        mbar_init(acc_full, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(Cfg::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // TMA of half stage q into ring slot q % 4 (issuer only)
    const uint32_t tx_bytes = (diag ? 1u : 2u) * Cfg::kRawF + (TWO ? 2u : 1u) * Cfg::kRawW;
    auto load_half = [&](int q) {
        const int64_t row = i0 + (int64_t)q * kGtHalf;
        const uint32_t dst = base + (q % kGtSlots) * Cfg::kRaw;
        mbar_expect_tx(raw_full(q), tx_bytes);
        tma_load_2d(dst, &tmF, (int)row, I * 128, raw_full(q));
        if (!diag) tma_load_2d(dst + Cfg::kRawF, &tmF, (int)row, J * 128, raw_full(q));
        bulk_g2s(dst + 2 * Cfg::kRawF, wa + row, Cfg::kRawW, raw_full(q));
        if (TWO) bulk_g2s(dst + 2 * Cfg::kRawF + Cfg::kRawW, wc + row, Cfg::kRawW, raw_full(q));
    };
    int loaded = 0;       // half stages whose TMA was issued (issuer)
    int last_half = -1;   // last half stage whose MMAs were committed (issuer)
    if (issuer) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmF)) : "memory");
        for (; loaded < kGtSlots && loaded < nq; ++loaded) load_half(loaded);
    }

    const int wq = wid & 3, hh = wid >> 2;
    const int m = 32 * wq + lane;                                  // accumulator row (TMEM lane)
    const uint32_t lane_off = (uint32_t)(32 * wq) << 16;
    // slicing items of this thread, the same in every half stage: rows
    // 4 ch .. 4 ch + 3 of the half (one 16-byte chunk of a raw column) of columns
    // cp[0], cp[1] of the I block (-> U) and of the J block (-> V).  A warp takes
    // the 8 chunks of columns {b, b+1, b+4, b+5}: its raw loads cover four whole
    // 128-byte column rows, and its 8-byte stores into the 128-byte swizzled
    // tiles meet each bank twice (the minimum for 256 bytes).
    const int ch = lane & 7;
    int cp[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int G = wid + 16 * p, cq = lane >> 3;                 // 32 groups of 4 columns
        cp[p] = 8 * (G >> 1) + 2 * (G & 1) + (cq & 1) + 4 * (cq >> 1);
    }
    const float tiny = 1.5f * 0x1p-100f;                            // columns past rank are zero
    float mu[2], ma[2], mc[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int ci = I * 128 + cp[p], cj = J * 128 + cp[p];
        mu[p] = ci < rank ? mag[ci] : tiny;
        ma[p] = cj < rank ? mag[rank + cj] : tiny;
        mc[p] = (TWO && cj < rank) ? mag[2 * rank + cj] : tiny;
    }
    const uint32_t d0 = tmem, d1 = tmem + NV;
    const uint32_t u_hi = sl, u_mid = sl + Cfg::kU, v_hi = sl + 2 * Cfg::kU, v_mid = v_hi + Cfg::kV;
    float run[CW];
#pragma unroll
    for (int e = 0; e < CW; ++e) run[e] = 0.f;
    bool ok = true;
    for (int q = 0; q < nq; ++q) {
        const int h = q & 1;                                       // slice half: rows 32 h .. 32 h + 31
        if (!mbar_wait_or_fail(raw_full(q), (uint32_t)(q / kGtSlots) & 1, &s_fail) ||
            (q >= 2 && !mbar_wait_or_fail(sl_empty(h), (uint32_t)((q >> 1) - 1) & 1, &s_fail))) {
            ok = false;
            break;
        }
        {
            const uint32_t rbase = base + (q % kGtSlots) * Cfg::kRaw;
            const uint32_t rJ0 = diag ? rbase : rbase + Cfg::kRawF;
            const uint32_t rW = rbase + 2 * Cfg::kRawF + 16 * ch;
            const int g = (ch >> 1) + 4 * h;                        // 8-row group in the 64-row slice stage
            const uint32_t ob = 8 * (ch & 1);                       // which 4 rows of the group
            const float4 one = make_float4(1.f, 1.f, 1.f, 1.f);
            const float4 w4 = lds4(rW);
            const float4 c4 = TWO ? lds4(rW + Cfg::kRawW) : one;
#pragma unroll 1
            for (int p = 0; p < 2; ++p) {
                const int c = p ? cp[1] : cp[0];
                const uint32_t off = (uint32_t)c * (kGtHalf * 4) + 16 * ch;
                const uint32_t o = swz(c, g) + ob, o2 = swz(128 + c, g) + ob;
                const float mup = p ? mu[1] : mu[0], map = p ? ma[1] : ma[0], mcp = p ? mc[1] : mc[0];
                slice4(lds4(rbase + off), one, mup, u_hi + o, u_mid + o);            // U = F(rows, I-block)
                const float4 xj = lds4(rJ0 + off);
                slice4(xj, w4, map, v_hi + o, v_mid + o);                             // wa F(rows, J-block)
                if (TWO) slice4(xj, c4, mcp, v_hi + o2, v_mid + o2);                 // wc F(rows, J-block)
            }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(sl_full(h));
            mbar_arrive(raw_empty(q));
        }
        const bool chunk_end = (q % kGtChunk) == kGtChunk - 1 || q == nq - 1;
        if (issuer) {
            // every warp has stored (and fenced) this half: issue its MMAs
            if (!mbar_wait_or_fail(sl_full(h), (uint32_t)(q >> 1) & 1, &s_fail)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const bool first = (q % kGtChunk) == 0;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint32_t off = 32u * (2 * h + j);
                const uint32_t acc = (first && j == 0) ? 0u : 1u;
                const uint64_t uh = sw128_desc(u_hi + off), um = sw128_desc(u_mid + off);
                const uint64_t vh = sw128_desc(v_hi + off), vm = sw128_desc(v_mid + off);
                umma_bf16(d0, uh, vh, kIdesc, acc);
                umma_bf16(d1, uh, vm, kIdesc, acc);
                umma_bf16(d1, um, vh, kIdesc, 1u);
                umma_bf16(d1, um, vm, kIdesc, 1u);
            }
            umma_commit(sl_empty(h));
            last_half = q;
            if (chunk_end) umma_commit(acc_full);
            if (loaded < nq) {
                // every warp has read raw half stage q: refill its slot with q + 4
                if (!mbar_wait_or_fail(raw_empty(q), (uint32_t)(q / kGtSlots) & 1, &s_fail)) {
                    ok = false;
                    break;
                }
                load_half(loaded++);
            }
        }
        if (chunk_end) {
            // drain the chunk: run += level 0 + level 1 over this thread's columns.  The
            // next chunk's first MMA is issued only after every warp has arrived on the
            // next half stage, which each does after these loads completed.
            __syncwarp();   // the issuer rejoins its warp: the TMEM loads are warp-collective
            if (!mbar_wait_or_fail(acc_full, (uint32_t)(q / kGtChunk) & 1, &s_fail)) {
                ok = false;
                break;
            }
            __syncwarp();
            tc_fence_after();
#pragma unroll
            for (int cb = 0; cb < CW / 16; ++cb) {
                uint32_t r0[16], r1[16];
                const uint32_t col = (uint32_t)(hh * CW + 16 * cb);
                tmem_ld16_async(tmem + lane_off + col, r0);
                tmem_ld16_async(tmem + lane_off + NV + col, r1);
                tmem_wait_ld32(r0, r1);
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    run[16 * cb + e] += __fadd_rn(__uint_as_float(r0[e]), __uint_as_float(r1[e]));
            }
            tc_fence_before();
        }
    }
    if (!ok) {
        s_fail = 1;
        atomicOr(flags, 4);
    } else {
        // this thread's row m of the tile: accumulator columns [hh CW, hh CW + CW), i.e.
        // Gram (hh CW) / 128, columns (hh CW) % 128 onwards; FP32 partials (the splits
        // are added in FP64)
        float* out = gpart + ((size_t)blockIdx.y * ntri + blockIdx.x) * 2 * 128 * 128;
        const int gsel = (hh * CW) / 128, c0 = (hh * CW) % 128;
        float* o = out + ((size_t)gsel * 128 + m) * 128 + c0;
#pragma unroll
        for (int e = 0; e < CW; e += 4)
            *reinterpret_cast<float4*>(o + e) = make_float4(run[e], run[e + 1], run[e + 2], run[e + 3]);
    }
    if (issuer) {
        // this CTA's copies and MMAs have completed before it exits (bounded waits;
        // immediate on the normal path)
        for (int j = loaded >= kGtSlots ? loaded - kGtSlots : 0; j < loaded; ++j)
            mbar_wait(raw_full(j), (uint32_t)(j / kGtSlots) & 1);
        if (last_half >= 0) mbar_wait(sl_empty(last_half & 1), (uint32_t)(last_half >> 1) & 1);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kCols) : "memory");
}

// Column maxima of |F|, |wa F| and |wc F| (as float bits, atomically maxed into
// cmax[0..rank), [rank..2 rank), [2 rank..3 rank); cmax zeroed beforehand).
// Block: 8 warps = 8 columns; blockIdx.y = row split of `per` rows.
__global__ void __launch_bounds__(256) k_colmax3(const float* __restrict__ F, int64_t ldf, int64_t N, int rank,
                                                 int64_t per, const float* __restrict__ wa,
                                                 const float* __restrict__ wc, unsigned* __restrict__ cmax) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (c >= rank) return;
    const int64_t i0 = (int64_t)blockIdx.y * per, i1 = min(i0 + per, N);
    const float* col = F + (int64_t)c * ldf;
    float mu = 0.f, ma = 0.f, mc = 0.f;
    int64_t i = i0 + 4 * lane;
    for (; i + 4 <= i1; i += 128) {
        const float4 x = *reinterpret_cast<const float4*>(col + i);
        const float4 a = *reinterpret_cast<const float4*>(wa + i);
        const float xv[4] = {x.x, x.y, x.z, x.w}, av[4] = {a.x, a.y, a.z, a.w};
        float cv[4] = {0.f, 0.f, 0.f, 0.f};
        if (wc) {
            const float4 q = *reinterpret_cast<const float4*>(wc + i);
            cv[0] = q.x; cv[1] = q.y; cv[2] = q.z; cv[3] = q.w;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            mu = fmaxf(mu, fabsf(xv[e]));
            ma = fmaxf(ma, fabsf(__fmul_rn(av[e], xv[e])));
            mc = fmaxf(mc, fabsf(__fmul_rn(cv[e], xv[e])));
        }
    }
    for (; i < i1; ++i) {   // the < 4 rows of the one lane whose next vector would cross i1
        const float x = col[i];
        mu = fmaxf(mu, fabsf(x));
        ma = fmaxf(ma, fabsf(__fmul_rn(wa[i], x)));
        if (wc) mc = fmaxf(mc, fabsf(__fmul_rn(wc[i], x)));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    if (lane == 0) {
        atomicMax(cmax + c, __float_as_uint(mu));
        atomicMax(cmax + rank + c, __float_as_uint(ma));
        atomicMax(cmax + 2 * rank + c, __float_as_uint(mc));
    }
}

// Magic number 1.5 * 2^(E + 16) per column, E the smallest integer with
// max < 2^E (frexp), so that (x + M) - M rounds x to the grid 2^(E - 7).
// Zero (or negligible, max < 2^-100) columns get the grid of 2^-100.
__global__ void k_magic(const unsigned* __restrict__ cmax, int n, float* __restrict__ mag) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const float mx = __uint_as_float(cmax[c]);
    int E = -100;
    if (mx >= 0x1p-100f) frexpf(mx, &E);
    mag[c] = ldexpf(1.5f, E + 16);
}

// Rows per split for the tensor-core Gram: a multiple of the 64-row slice stage, at
// least 4,096 rows unless N is smaller, the split count chosen so that
// ntri x nsplit CTAs fill whole waves of one CTA per SM.
int64_t gram_tc_per(int64_t N, int64_t ntri, int nsm, int* nsplit) {
    int64_t best_per = (N + 63) / 64 * 64;
    double best_eff = -1.0;
    for (int64_t sp = 1; sp <= 64; ++sp) {
        const int64_t pr = ((N + sp - 1) / sp + 63) / 64 * 64;
        if (sp > 1 && pr < 4096) break;
        const int64_t ns = (N + pr - 1) / pr, blocks = ntri * ns;
        const double eff = (double)blocks / (double)(((blocks + nsm - 1) / nsm) * nsm);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best_per = pr;
        }
    }
    *nsplit = (int)((N + best_per - 1) / best_per);
    return best_per;
}

bool gram_tc_eligible(const float* F, int64_t ldf, int64_t N, int rank) {
    if (const char* e = getenv("KEVD_GRAM")) {
        if (e[0] == 'f') return false;                          // KEVD_GRAM=ffma: the FFMA kernel
    }
    return rank >= 1 && N >= 1 && N < ((int64_t)1 << 31) && ldf % 4 == 0 &&
           (reinterpret_cast<uintptr_t>(F) % 16) == 0 && (uint64_t)ldf * 4 < ((uint64_t)1 << 40);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

cudaError_t launch_gram_tc(const float* F, int64_t ldf, int64_t N, int rank, const float* wa, const float* wc,
                           unsigned* cmax, float* mag, float* gpart, int* flags, int nb, int ntri, int64_t per,
                           int nsplit, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(cmax, 0, 3 * (size_t)rank * sizeof(unsigned), s)) != cudaSuccess) return e;
    {
        const int ncs = (int)std::max<int64_t>(1, std::min<int64_t>(64, N / 8192));
        const int64_t pr = ((N + ncs - 1) / ncs + 127) / 128 * 128;
        k_colmax3<<<dim3((rank + 7) / 8, (unsigned)((N + pr - 1) / pr)), 256, 0, s>>>(F, ldf, N, rank, pr, wa, wc,
                                                                                       cmax);
        k_magic<<<(3 * rank + 255) / 256, 256, 0, s>>>(cmax, 3 * rank, mag);
    }
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)rank};
    const cuuint64_t strides[1] = {(cuuint64_t)ldf * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kGtHalf, 128};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(F), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const dim3 grid((unsigned)ntri, (unsigned)nsplit);
    if (wc) {
        const size_t smem = GtCfg<true>::kSmem;
        if ((e = cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_gram_tc<true><<<grid, kGtThreads, smem, s>>>(map, wa, wc, mag, rank, N, nb, per, gpart, ntri, flags);
    } else {
        const size_t smem = GtCfg<false>::kSmem;
        if ((e = cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_gram_tc<false><<<grid, kGtThreads, smem, s>>>(map, wa, nullptr, mag, rank, N, nb, per, gpart, ntri, flags);
    }
    return cudaGetLastError();
}

}  // namespace kevd
