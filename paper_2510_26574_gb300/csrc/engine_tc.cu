// Kernel-column engine of the precision form on the 5th-generation tensor
// cores (tcgen05 / TMEM), Algorithm 2's G = (K(:,S) - F F(S,:)^T) L^-T.
//
// Operands are split into BF16 hi/lo halves (v = hi + lo, hi = bf16(v),
// lo = bf16(v - hi)) and each product is formed as hi*hi + hi*lo + lo*hi with
// FP32 accumulation in TMEM (UMMA kind::f16, M = 128 rows, N = BN pivots,
// K = 16 per instruction).  Two accumulators per tile:
//   D_x = X(i,:) . X(s,:)      (the norm expansion's cross term)
//   D_f = F(i,:k) . F(s,:k)
// and the epilogue forms R = exp(-(|x_i|^2 + |x_s|^2 - 2 D_x)/eps) - D_f in
// FP32, solves G L^T = R by blocked forward substitution in FP32 (16-column
// diagonal solves, trailing updates spread over all threads, L staged in
// shared memory by one bulk copy), writes G into F(:, k:k+m), and updates the
// FP64 residual diagonal and the per-64-row tile statistics of the next
// round's sampler.  (A tensor-core solve with an explicit BF16-split L^-1 was
// measured to lose ~1.5 digits on late pivots, so the solve stays in FP32.)
//
// Data movement per 64-wide K chunk: the pivot panel (pre-split, pre-swizzled
// by k_panel, L2-resident) arrives by one bulk async copy completing on an
// mbarrier, issued one chunk ahead so that its L2 latency overlaps the
// previous chunk; the 128 x 64 FP32 slice of X or F is loaded by all threads one
// chunk ahead (register prefetch), split and stored in the 128-byte-swizzled
// K-major layout; one elected thread issues the 12 MMAs and commits them to
// the stage's mbarrier.  Two stages.  Every wait is bounded (about one
// second); on a timeout the CTA records an error, waits (bounded) for its own
// copies and MMAs, frees its TMEM and exits.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "common.cuh"
#include "factor.cuh"
#include "tc_ptx.cuh"

namespace kevd {

// bar.red.or on named barrier `id` over `nthreads` threads: every participant
// gets the OR of `pred` (a uniform decision for a group of warps).
static __device__ __forceinline__ bool named_bar_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}


// ---------------------------------------------------------------------------
// Pivot panel of the round: X(S,:) and F(S,:k) of the m accepted pivots, split
// into hi/lo bf16 in the engine's swizzled K-major layout (zero rows past m,
// zero K past d or k), plus FP32 norms and pivot rows.  Block c = chunk c.
// ---------------------------------------------------------------------------
template <int BN>
__global__ void __launch_bounds__(256) k_panel(FactorWs w, PanelWs p, int d, int b) {
    const FactorState* st = w.st;
    if (st->done || st->m == 0) return;
    const int k = st->k, m = st->m;
    const int nx = (d + kTcBK - 1) / kTcBK;
    const int c = blockIdx.x;
    if (c >= nx + (k + kTcBK - 1) / kTcBK) return;
    uint8_t* hi = reinterpret_cast<uint8_t*>(p.panel) + (size_t)(2 * c) * BN * 128;
    uint8_t* lo = hi + (size_t)BN * 128;
    for (int u = threadIdx.x; u < BN * 8; u += blockDim.x) {
        const int l = u >> 3, g = u & 7;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float x = 0.f;
            if (l < m) {
                const int pos = w.acc_pos[l];
                if (c < nx) {
                    const int col = c * kTcBK + g * 8 + e;
                    if (col < d) x = (float)w.XSP[(size_t)col * b + pos];
                } else {
                    const int col = (c - nx) * kTcBK + g * 8 + e;
                    if (col < k) x = (float)w.FSP[(size_t)col * b + pos];
                }
            }
            v[e] = x;
        }
        split_store8(v, hi + swz(l, g), lo + swz(l, g));
    }
    if (c == 0) {
        for (int l = threadIdx.x; l < BN; l += blockDim.x) {
            p.nS[l] = l < m ? (float)w.xnS[w.acc_pos[l]] : 0.f;
            p.pidx[l] = l < m ? w.prop[w.acc_pos[l]] : -1;
        }
    }
}

// ---------------------------------------------------------------------------
// L(T,T) in FP32 (BN x BN, zero past m) for the engine's forward substitution.
// ---------------------------------------------------------------------------
template <int BN>
__global__ void k_lprep(FactorWs w, PanelWs p, int b) {
    const FactorState* st = w.st;
    if (st->done || st->m == 0) return;
    const int m = st->m;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < BN * BN; e += gridDim.x * blockDim.x) {
        const int a = e / BN, a2 = e % BN;
        p.Lf[e] = (a < m && a2 <= a) ? (float)w.Lc[(size_t)a * b + a2] : 0.f;
    }
}

// ---------------------------------------------------------------------------
// The engine: a persistent, warp-specialised kernel, one CTA per SM, which
// walks the 128-row tiles blockIdx.x, blockIdx.x + gridDim.x, ...
//   warps 0-7  (producers): load the 128 x 64 FP32 slice of X or F of each K
//              chunk (two chunks ahead in registers), split it into BF16 hi/lo,
//              store it in the swizzled K-major layout of a ring stage and
//              arrive on a_full[stage] (one arrival per warp);
//   warp 12    (panel): copies the pre-split pivot panel of the chunk into the
//              stage by one bulk async copy completing on b_full[stage];
//   warp 13    (MMA): allocates TMEM, issues the 12 MMAs of each chunk into
//              the tile's accumulator pair (D_x, D_f) in one of two TMEM
//              buffers, commits each chunk to empty[stage] and each finished
//              tile to tmem_full[buffer];
//   warps 8-11 (epilogue, thread = tile row, warp % 4 = TMEM lane quarter):
//              R = exp(-(n_i + n_s - 2 D_x)/eps) - D_f written back over D_x,
//              then G L^T = R solved in place in TMEM by 16-column blocks
//              (diagonal solve in registers, trailing columns updated through
//              TMEM loads/stores, L from shared memory by broadcast reads), G
//              written to F(:, k:k+m), the buffer released to the MMA warp
//              (tmem_empty), then the FP64 residual diagonal and the per-64-row
//              tile statistics of the next round's sampler.
// While the epilogue works on tile t, the producers and the MMA warp already
// run tile t+1 into the other TMEM buffer.  Every wait is bounded (about one
// second) and also ends when another role of the CTA has failed; a failing CTA
// records the error, waits (bounded) for its own copies and MMAs, frees its
// TMEM and exits.
// ---------------------------------------------------------------------------
template <int BN>
struct EngineCfg {
    static constexpr int kStages = BN == 128 ? 2 : (BN == 64 ? 4 : 5);   // ring stages that fit with L
    static constexpr uint32_t kAbytes = kTcBM * 128;                    // one 128 x 64 bf16 tile
    static constexpr uint32_t kBbytes = BN * 128;
    static constexpr uint32_t kStage = 2 * kAbytes + 2 * kBbytes;
    static constexpr uint32_t kLbytes = BN * BN * 4;
    static constexpr uint32_t kCols = 4 * BN;                           // 2 buffers x (D_x, D_f)
    static constexpr size_t kSmem = (size_t)kStages * kStage + kLbytes + 1024;
};

constexpr int kProdWarps = 8, kEpiWarp0 = 8, kPanelWarp = 12, kMmaWarp = 13;
constexpr int kEngineThreads = 14 * 32;

template <int BN>
__global__ void __launch_bounds__(kEngineThreads, 1)
    k_engine_tc(FactorWs w, PanelWs p, const float* __restrict__ X, float* __restrict__ F, int64_t ldf,
                double* __restrict__ rho, int64_t N, int d, float inv_eps) {
    using Cfg = EngineCfg<BN>;
    constexpr int S = Cfg::kStages;
    constexpr uint32_t kAbytes = Cfg::kAbytes, kBbytes = Cfg::kBbytes, kStage = Cfg::kStage;
    constexpr uint32_t kIdesc = idesc_bf16(kTcBM, BN);
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[3 * S + 5];   // a_full[S], b_full[S], empty[S], tmem_full[2], tmem_empty[2], L
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_fail;
    __shared__ float s_dinv[BN], s_nS[BN];
    __shared__ int64_t s_pidx[BN];
    __shared__ double red_s[2][4], red_m[2][4];
    __shared__ int64_t red_i[2][4];

    const FactorState* st = w.st;
    if (st->done) return;
    const int m = st->m;
    if (m == 0) return;
    const int k = st->k;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t ntiles = (N + kTcBM - 1) / kTcBM;
    const int nx = (d + kTcBK - 1) / kTcBK;
    const int nf = (k + kTcBK - 1) / kTcBK;
    const int nchunks = nx + nf;
    const int my_tiles = (int)((ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x);

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sm = smem_raw + (base - raw);
    const uint32_t lbase = base + S * kStage;
    const float* Ls = reinterpret_cast<const float*>(sm + S * kStage);
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto a_full = [&](int s) { return bar0 + 8u * s; };
    auto b_full = [&](int s) { return bar0 + 8u * (S + s); };
    auto empty = [&](int s) { return bar0 + 8u * (2 * S + s); };
    auto tmem_full = [&](int b) { return bar0 + 8u * (3 * S + b); };
    auto tmem_empty = [&](int b) { return bar0 + 8u * (3 * S + 2 + b); };
    const uint32_t bar_L = bar0 + 8u * (3 * S + 4);
    auto fail_now = [&]() {
        s_fail = 1;
        atomicExch(p.err, 1);
    };

    if (tid == 0) {
        for (int s2 = 0; s2 < S; ++s2) {
            mbar_init(a_full(s2), kProdWarps);
            mbar_init(b_full(s2), 1);
            mbar_init(empty(s2), 1);
        }
        for (int b2 = 0; b2 < 2; ++b2) {
            mbar_init(tmem_full(b2), 1);
            mbar_init(tmem_empty(b2), 4);
        }
        mbar_init(bar_L, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (wid == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(Cfg::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (wid < kProdWarps) {
        // ---------------- producers ----------------
        const int lrow = 32 * (wid & 3) + lane;   // tile row loaded by this thread
        const int gbase = wid >> 2;              // 8-element groups gbase, gbase + 2, + 4, + 6
        const bool xvec = (d % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
        // flat chunk sequence g = it * nchunks + c over this CTA's tiles; two chunks
        // of loads stay in flight (register double buffer, unrolled by two so
        // that both buffers keep compile-time indices)
        auto load_chunk = [&](int gg, float (&v)[4][8]) {
            const int it = gg / nchunks, c = gg - it * nchunks;
            const int64_t grow = (int64_t)(blockIdx.x + (int64_t)it * gridDim.x) * kTcBM + lrow;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int g8 = gbase + 2 * t;
                if (c < nx) {
                    const int col = c * kTcBK + g8 * 8;
                    if (grow < N && xvec && col + 8 <= d) {
                        const float4 a = __ldg(reinterpret_cast<const float4*>(X + grow * d + col));
                        const float4 bq = __ldg(reinterpret_cast<const float4*>(X + grow * d + col + 4));
                        v[t][0] = a.x; v[t][1] = a.y; v[t][2] = a.z; v[t][3] = a.w;
                        v[t][4] = bq.x; v[t][5] = bq.y; v[t][6] = bq.z; v[t][7] = bq.w;
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[t][e] = (grow < N && col + e < d) ? X[grow * d + col + e] : 0.f;
                    }
                } else {
                    const int col = (c - nx) * kTcBK + g8 * 8;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        v[t][e] = (grow < N && col + e < k) ? __ldg(F + (int64_t)(col + e) * ldf + grow) : 0.f;
                }
            }
        };
        const int total = my_tiles * nchunks;
        bool ok = true;
        auto step = [&](int g, float (&v)[4][8]) {
            const int s2 = g % S;
            const uint32_t use = (uint32_t)(g / S);
            if (g >= S && !mbar_wait_sleep(empty(s2), (use - 1) & 1, &s_fail, 64)) {
                ok = false;
                return;
            }
            uint8_t* A_hi = sm + s2 * kStage;
            uint8_t* A_lo = A_hi + kAbytes;
#pragma unroll
            for (int t = 0; t < 4; ++t) split_store8(v[t], A_hi + swz(lrow, gbase + 2 * t), A_lo + swz(lrow, gbase + 2 * t));
            if (g + 2 < total) load_chunk(g + 2, v);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(a_full(s2));
        };
        float va[4][8], vb[4][8];
        if (total > 0) load_chunk(0, va);
        if (total > 1) load_chunk(1, vb);
        for (int g = 0; g < total && ok; g += 2) {
            step(g, va);
            if (ok && g + 1 < total) step(g + 1, vb);
        }
        if (!ok) fail_now();
    } else if (wid == kPanelWarp) {
        // ---------------- pivot panel copies (one lane) ----------------
        if (lane == 0) {
            mbar_expect_tx(bar_L, Cfg::kLbytes);
            bulk_g2s(lbase, p.Lf, Cfg::kLbytes, bar_L);
            bool ok = true;
            int g = 0;
            for (int it = 0; it < my_tiles && ok; ++it) {
                for (int c = 0; c < nchunks; ++c, ++g) {
                    const int s2 = g % S;
                    const uint32_t use = (uint32_t)(g / S);
                    if (g >= S && !mbar_wait_sleep(empty(s2), (use - 1) & 1, &s_fail, 64)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(b_full(s2), 2 * kBbytes);
                    bulk_g2s(base + s2 * kStage + 2 * kAbytes,
                             reinterpret_cast<const uint8_t*>(p.panel) + (size_t)(2 * c) * kBbytes, 2 * kBbytes,
                             b_full(s2));
                }
            }
            if (!ok) fail_now();
            // every copy of this CTA has landed before it exits (bounded; immediate on the normal path)
            mbar_wait(bar_L, 0);
            for (int j = g - S; j < g; ++j)
                if (j >= 0) mbar_wait(b_full(j % S), (uint32_t)(j / S) & 1);
        }
    } else if (wid == kMmaWarp) {
        // ---------------- MMA issue (one lane) ----------------
        if (lane == 0) {
            bool ok = true;
            int g = 0, issued = 0;
            for (int it = 0; it < my_tiles && ok; ++it) {
                const int buf = it & 1;
                if (it >= 2 && !mbar_wait_sleep(tmem_empty(buf), (uint32_t)((it >> 1) - 1) & 1, &s_fail, 64)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tdx = tmem + (uint32_t)(buf * 2 * BN), tdf = tdx + BN;
                for (int c = 0; c < nchunks; ++c, ++g) {
                    const int s2 = g % S;
                    const uint32_t use = (uint32_t)(g / S);
                    if (!mbar_wait_or_fail(a_full(s2), use & 1, &s_fail) ||
                        !mbar_wait_or_fail(b_full(s2), use & 1, &s_fail)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = c < nx ? tdx : tdf;
                    const bool first = (c == 0) || (c == nx);
                    const uint32_t a_hi = base + s2 * kStage, a_lo = a_hi + kAbytes;
                    const uint32_t b_hi = a_hi + 2 * kAbytes, b_lo = b_hi + kBbytes;
#pragma unroll
                    for (int j = 0; j < kTcBK / 16; ++j) {
                        const uint32_t off = 32u * j;
                        const uint64_t ah = sw128_desc(a_hi + off), al = sw128_desc(a_lo + off);
                        const uint64_t bh = sw128_desc(b_hi + off), bl = sw128_desc(b_lo + off);
                        umma_bf16(dt, ah, bh, kIdesc, (first && j == 0) ? 0u : 1u);
                        umma_bf16(dt, ah, bl, kIdesc, 1u);
                        umma_bf16(dt, al, bh, kIdesc, 1u);
                    }
                    umma_commit(empty(s2));
                    issued = g + 1;
                }
                if (ok) umma_commit(tmem_full(buf));
            }
            if (!ok) fail_now();
            // all MMAs of this CTA complete before its TMEM is freed (the last commit covers the earlier ones)
            if (issued > 0) {
                const int j = issued - 1;
                mbar_wait(empty(j % S), (uint32_t)(j / S) & 1);
            }
        }
    } else {
        // ---------------- epilogue: warps 8-11, thread = tile row ----------------
        const int q = wid & 3;
        const int et = tid - kEpiWarp0 * 32;
        const int row = 32 * q + lane;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        bool bad = !mbar_wait_or_fail(bar_L, 0, &s_fail);
        for (int l = et; l < BN; l += 128) {
            s_nS[l] = p.nS[l];
            s_pidx[l] = p.pidx[l];
            s_dinv[l] = (!bad && l < m) ? 1.f / Ls[l * BN + l] : 0.f;
        }
        bool ok = !named_bar_or(1, 128, bad);
        for (int it = 0; it < my_tiles && ok; ++it) {
            const int buf = it & 1;
            const int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
            const int64_t grow = tile * kTcBM + row;
            bad = !mbar_wait_sleep(tmem_full(buf), (uint32_t)(it >> 1) & 1, &s_fail, 64);
            if (named_bar_or(1, 128, bad)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t tx0 = tmem + (uint32_t)(buf * 2 * BN) + lane_off, tf0 = tx0 + BN;
            // R = exp(-(n_i + n_s - 2 D_x)/eps) - D_f, written back over D_x; the
            // TMEM loads of the next 16-column block are in flight while one is computed
            const float ni = grow < N ? (float)w.xn[grow] : 0.f;
            auto r_block = [&](int c0, const uint32_t (&xr)[16], const uint32_t (&fr)[16]) {
                float rr[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int l = c0 + e;
                    float kv = 0.f;
                    if (l < m) {
                        if (s_pidx[l] == grow) {
                            kv = 1.f;
                        } else {
                            const float d2 = fmaxf(ni + s_nS[l] - 2.f * __uint_as_float(xr[e]), 0.f);
                            kv = expf(-d2 * inv_eps);
                        }
                    }
                    rr[e] = l < m ? kv - (nf > 0 ? __uint_as_float(fr[e]) : 0.f) : 0.f;
                }
                tmem_st16(tx0 + c0, rr);
            };
            {
                uint32_t xa[16], fa[16], xb[16], fb[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) fa[e] = fb[e] = 0u;
                tmem_ld16_async(tx0, xa);
                if (nf > 0) tmem_ld16_async(tf0, fa);
                tmem_wait_ld32(xa, fa);
                for (int c0 = 0; c0 < m; c0 += 32) {
                    const bool hb = c0 + 16 < m;
                    if (hb) {
                        tmem_ld16_async(tx0 + c0 + 16, xb);
                        if (nf > 0) tmem_ld16_async(tf0 + c0 + 16, fb);
                    }
                    r_block(c0, xa, fa);
                    if (hb) {
                        tmem_wait_ld32(xb, fb);
                        if (c0 + 32 < m) {
                            tmem_ld16_async(tx0 + c0 + 32, xa);
                            if (nf > 0) tmem_ld16_async(tf0 + c0 + 32, fa);
                        }
                        r_block(c0 + 16, xb, fb);
                        if (c0 + 32 < m) tmem_wait_ld32(xa, fa);
                    }
                }
            }
            tmem_wait_st();
            // G L^T = R by 16-column blocks, in place in TMEM: diagonal block solved in
            // registers, the trailing blocks updated two at a time with the next two loads
            // in flight
            float nrm = 0.f;
            for (int jb = 0; jb < m; jb += 16) {
                uint32_t gr[16], ta[16], tb[16];
                const int c1 = jb + 16, c2 = jb + 32;
                tmem_ld16_async(tx0 + jb, gr);
                if (c1 < m) tmem_ld16_async(tx0 + c1, ta);
                if (c2 < m) tmem_ld16_async(tx0 + c2, tb);
                tmem_wait_ld16(gr);
                tmem_wait_ld32(ta, tb);
                float gv[16];
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) gv[jj] = __uint_as_float(gr[jj]);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const float* Lj = Ls + (jb + jj) * BN + jb;
                    float acc = gv[jj];
#pragma unroll
                    for (int ll = 0; ll < jj; ++ll) acc = fmaf(-Lj[ll], gv[ll], acc);
                    gv[jj] = (jb + jj < m) ? acc * s_dinv[jb + jj] : 0.f;
                }
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    nrm = fmaf(gv[jj], gv[jj], nrm);
                    if (grow < N && jb + jj < m) F[(int64_t)(k + jb + jj) * ldf + grow] = gv[jj];
                }
                auto update = [&](int cb, const uint32_t (&tr)[16]) {
                    float tv[16];
#pragma unroll
                    for (int cc = 0; cc < 16; ++cc) {
                        const float4* Lr = reinterpret_cast<const float4*>(Ls + (cb + cc) * BN + jb);
                        float acc = __uint_as_float(tr[cc]);
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float4 lv = Lr[u];
                            acc = fmaf(-lv.x, gv[4 * u], acc);
                            acc = fmaf(-lv.y, gv[4 * u + 1], acc);
                            acc = fmaf(-lv.z, gv[4 * u + 2], acc);
                            acc = fmaf(-lv.w, gv[4 * u + 3], acc);
                        }
                        tv[cc] = acc;
                    }
                    tmem_st16(tx0 + cb, tv);
                };
                for (int cb = c1; cb < m; cb += 32) {
                    update(cb, ta);
                    if (cb + 32 < m) tmem_ld16_async(tx0 + cb + 32, ta);
                    if (cb + 16 < m) update(cb + 16, tb);
                    if (cb + 48 < m) tmem_ld16_async(tx0 + cb + 48, tb);
                    if (cb + 32 < m) tmem_wait_ld32(ta, tb);
                }
                tmem_wait_st();
            }
            // TMEM buffer back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tmem_empty(buf));
            // FP64 residual diagonal and the per-64-row tile statistics
            double rnew = 0.0, rmax = -1.0;
            int64_t ridx = LLONG_MAX;
            if (grow < N) {
                rnew = fmax(rho[grow] - (double)nrm, 0.0);
                rho[grow] = rnew;
                rmax = rnew;
                ridx = grow;
            }
            const double sum = warp_sum(rnew);
            warp_argmax(rmax, ridx);
            const int pb = it & 1;
            if (lane == 0) {
                red_s[pb][q] = sum;
                red_m[pb][q] = rmax;
                red_i[pb][q] = ridx;
            }
            named_bar_or(1, 128, false);
            if (et < 2) {
                const int64_t t2 = 2 * tile + et;
                if (t2 * kBM < N) {
                    double tm = red_m[pb][2 * et];
                    int64_t ti = red_i[pb][2 * et];
                    argmax_merge(tm, ti, red_m[pb][2 * et + 1], red_i[pb][2 * et + 1]);
                    w.tile_sum[t2] = red_s[pb][2 * et] + red_s[pb][2 * et + 1];
                    w.tile_max[t2] = tm;
                    w.tile_idx[t2] = ti;
                }
            }
        }
        if (!ok) fail_now();
    }

    // all roles done: free TMEM
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (wid == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kCols) : "memory");
}

template <int BN>
static cudaError_t launch_bn(const FactorWs& w, const PanelWs& p, const float* X, float* F, int64_t ldf, double* rho,
                             int64_t N, int d, int b, double inv_eps, int r, cudaStream_t s) {
    const int nch = tc_chunks(d, r);
    k_panel<BN><<<nch, 256, 0, s>>>(w, p, d, b);
    k_lprep<BN><<<(BN * BN + 255) / 256, 256, 0, s>>>(w, p, b);
    const size_t smem = EngineCfg<BN>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(k_engine_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t ntiles = (N + kTcBM - 1) / kTcBM;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, nsm));
    k_engine_tc<BN><<<grid, kEngineThreads, smem, s>>>(w, p, X, F, ldf, rho, N, d, (float)inv_eps);
    return cudaGetLastError();
}

cudaError_t launch_engine_tc(const FactorWs& w, const PanelWs& p, const float* X, float* F, int64_t ldf, double* rho,
                             int64_t N, int d, int b, double inv_eps, int r, cudaStream_t s) {
    if (b <= 32) return launch_bn<32>(w, p, X, F, ldf, rho, N, d, b, inv_eps, r, s);
    if (b <= 64) return launch_bn<64>(w, p, X, F, ldf, rho, N, d, b, inv_eps, r, s);
    return launch_bn<128>(w, p, X, F, ldf, rho, N, d, b, inv_eps, r, s);
}

}  // namespace kevd
