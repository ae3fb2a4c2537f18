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

#include "common.cuh"
#include "factor.cuh"
#include "tc_ptx.cuh"

namespace kevd {


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
// The engine: one CTA per 128-row tile, 256 threads.
// ---------------------------------------------------------------------------
template <int BN>
__global__ void __launch_bounds__(256, 1) k_engine_tc(FactorWs w, PanelWs p, const float* __restrict__ X,
                                                      float* __restrict__ F, int64_t ldf, double* __restrict__ rho,
                                                      int64_t N, int d, float inv_eps) {
    constexpr uint32_t kAbytes = kTcBM * 128;           // one 128 x 64 bf16 tile
    constexpr uint32_t kBbytes = BN * 128;
    constexpr uint32_t kStage = 2 * kAbytes + 2 * kBbytes;
    constexpr uint32_t kLbytes = BN * BN * 4;           // L in FP32
    constexpr uint32_t kCols = 2 * BN;                  // D_x, D_f
    constexpr uint32_t kIdesc = idesc_bf16(kTcBM, BN);
    constexpr int TB = 16;                              // column block of the forward substitution
    static_assert(kTcBM * (BN + 1) * 4 <= 2 * kStage, "R tile must fit in the stage buffers");
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[5];           // [0,1] panel, [2,3] MMA, [4] L
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail, s_issued, s_bissued;
    __shared__ double red[8];
    __shared__ double redm[8];
    __shared__ int64_t redi[8];

    const FactorState* st = w.st;
    if (st->done) return;
    const int m = st->m;
    if (m == 0) return;
    const int k = st->k;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * kTcBM;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sm = smem_raw + (base - raw);
    const uint32_t lbase = base + 2 * kStage;
    const uint32_t bar_b0 = smem_u32(&bars[0]), bar_m0 = smem_u32(&bars[2]);
    const uint32_t bar_L = smem_u32(&bars[4]);
    const float* Ls = reinterpret_cast<const float*>(sm + 2 * kStage);

    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(smem_u32(&bars[i]), 1);
        s_fail = 0;
        s_issued = 0;
        s_bissued = 0;
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
    const uint32_t tmem_x = tmem, tmem_f = tmem + BN;
    if (tid == 0) {   // L for the forward substitution, needed only after the main loop
        mbar_expect_tx(bar_L, kLbytes);
        bulk_g2s(lbase, p.Lf, kLbytes, bar_L);
    }

    const int nx = (d + kTcBK - 1) / kTcBK;
    const int nf = (k + kTcBK - 1) / kTcBK;
    const int nchunks = nx + nf;
    const bool xvec = (d % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    // loader mapping: row = 32*(wid%4) + lane, 8-element groups (wid/4) + 2t, t = 0..3
    const int lrow = 32 * (wid & 3) + lane;
    const int64_t grow = row0 + lrow;
    const int gbase = wid >> 2;
    bool fail = false;

    float v[4][8];
    auto load_chunk = [&](int c) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int g = gbase + 2 * t;
            if (c < nx) {
                const int col = c * kTcBK + g * 8;
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
                const int col = (c - nx) * kTcBK + g * 8;
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[t][e] = (grow < N && col + e < k) ? __ldg(F + (int64_t)(col + e) * ldf + grow) : 0.f;
            }
        }
    };

    // the pivot panel of chunk c is copied one chunk ahead: chunks 0 and 1 here,
    // chunk c + 1 by thread 0 right after issuing the MMAs of chunk c (once the
    // MMAs of chunk c - 1 have released that stage)
    auto issue_panel = [&](int c) {
        const int s = c & 1;
        mbar_expect_tx(bar_b0 + 8 * s, 2 * kBbytes);
        bulk_g2s(base + s * kStage + 2 * kAbytes, reinterpret_cast<const uint8_t*>(p.panel) + (size_t)(2 * c) * kBbytes,
                 2 * kBbytes, bar_b0 + 8 * s);
        s_bissued = c + 1;
    };
    if (tid == 0) {
        issue_panel(0);
        if (nchunks > 1) issue_panel(1);
    }
    load_chunk(0);
    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        const uint32_t use = (uint32_t)(c >> 1);
        uint8_t* A_hi = sm + s * kStage;
        uint8_t* A_lo = A_hi + kAbytes;
        const uint32_t B_s = base + s * kStage + 2 * kAbytes;
        // stage s is free once the MMAs of chunk c-2 completed
        if (c >= 2 && !fail) fail = !mbar_wait(bar_m0 + 8 * s, (use - 1) & 1);
        if (__syncthreads_or(fail)) {
            fail = true;
            break;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int g = gbase + 2 * t;
            split_store8(v[t], A_hi + swz(lrow, g), A_lo + swz(lrow, g));
        }
        if (c + 1 < nchunks) load_chunk(c + 1);   // in flight during the barrier and the MMA issue
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait(bar_b0 + 8 * s, use & 1)) {
                s_fail = 1;
                fail = true;
            } else {
                tc_fence_after();
                const uint32_t dt = c < nx ? tmem_x : tmem_f;
                const bool first = (c == 0) || (c == nx);
                const uint32_t a_hi = base + s * kStage, a_lo = a_hi + kAbytes;
                const uint32_t b_hi = B_s, b_lo = B_s + kBbytes;
#pragma unroll
                for (int j = 0; j < kTcBK / 16; ++j) {
                    const uint32_t off = 32u * j;
                    const uint64_t ah = sw128_desc(a_hi + off), al = sw128_desc(a_lo + off);
                    const uint64_t bh = sw128_desc(b_hi + off), bl = sw128_desc(b_lo + off);
                    umma_bf16(dt, ah, bh, kIdesc, (first && j == 0) ? 0u : 1u);
                    umma_bf16(dt, ah, bl, kIdesc, 1u);
                    umma_bf16(dt, al, bh, kIdesc, 1u);
                }
                umma_commit(bar_m0 + 8 * s);
                s_issued = c + 1;
                if (c + 1 < nchunks && c + 1 >= 2) {
                    // stage s^1 holds chunk c-1 until its MMAs complete
                    if (!mbar_wait(bar_m0 + 8 * (s ^ 1), (uint32_t)((c - 1) >> 1) & 1)) {
                        s_fail = 1;
                        fail = true;
                    } else {
                        issue_panel(c + 1);
                    }
                }
            }
        }
    }
    // all MMAs complete: the last commit covers every earlier MMA of thread 0
    if (__syncthreads_or(fail)) fail = true;
    if (s_issued > 0) {
        const int cl = s_issued - 1;
        if (!mbar_wait(bar_m0 + 8 * (cl & 1), (uint32_t)(cl >> 1) & 1)) fail = true;
    }
    if (__syncthreads_or(fail)) fail = true;
    tc_fence_after();

    const int q = wid & 3, h = wid >> 2;
    const int erow = 32 * q + lane;
    const int64_t egrow = row0 + erow;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    float* Rs = reinterpret_cast<float*>(sm);   // 128 x (BN+1), reuses the stage buffers
    if (!fail) {
        // ---- epilogue 1: R = exp(-(n_i + n_s - 2 D_x)/eps) - D_f -> shared memory ----
        const float ni = egrow < N ? (float)w.xn[egrow] : 0.f;
        for (int c0 = h * (BN / 2); c0 < (h + 1) * (BN / 2); c0 += 16) {
            float dx[16], df[16];
            tmem_ld16(tmem_x + lane_off + c0, dx);
            if (nf > 0) {
                tmem_ld16(tmem_f + lane_off + c0, df);
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) df[e] = 0.f;
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int l = c0 + e;
                float kv = 0.f;
                if (l < m) {
                    if (p.pidx[l] == egrow) {
                        kv = 1.f;
                    } else {
                        const float d2 = fmaxf(ni + p.nS[l] - 2.f * dx[e], 0.f);
                        kv = expf(-d2 * inv_eps);
                    }
                }
                Rs[erow * (BN + 1) + l] = kv - df[e];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    if (!fail && tid == 0 && !mbar_wait(bar_L, 0)) s_fail = 1;
    __syncthreads();
    if (s_fail) fail = true;
    if (fail) {
        if (tid == 0) {
            mbar_wait(bar_L, 0);   // bounded: the L copy may still be in flight
            for (int j = s_bissued - 2; j < s_bissued; ++j)   // and the last panel copy of each stage
                if (j >= 0) mbar_wait(bar_b0 + 8 * (j & 1), (uint32_t)(j >> 1) & 1);
            atomicExch(p.err, 1);
        }
        return;
    }

    // ---- epilogue 2: G L^T = R by blocked forward substitution (FP32) ----
    {
        const int srow = tid & (kTcBM - 1), half = tid >> 7;
        float* Ri = Rs + srow * (BN + 1);
        for (int jb = 0; jb < m; jb += TB) {
            const int je = min(jb + TB, m);
            if (half == 0) {   // diagonal block: one thread per row
                for (int j = jb; j < je; ++j) {
                    const float* Lj = Ls + j * BN;
                    float s0 = Ri[j], s1 = 0.f;
                    int l = jb;
                    for (; l + 1 < j; l += 2) {
                        s0 = fmaf(-Lj[l], Ri[l], s0);
                        s1 = fmaf(-Lj[l + 1], Ri[l + 1], s1);
                    }
                    if (l < j) s0 = fmaf(-Lj[l], Ri[l], s0);
                    Ri[j] = (s0 + s1) / Lj[j];
                }
            }
            __syncthreads();
            if (je < m) {      // trailing columns: R(:, c) -= G(:, jb:je) L(c, jb:je)^T
                float g[TB];
#pragma unroll
                for (int t = 0; t < TB; ++t) g[t] = jb + t < je ? Ri[jb + t] : 0.f;
                for (int c = je + half; c < m; c += 2) {
                    const float4* Lc4 = reinterpret_cast<const float4*>(Ls + c * BN + jb);
                    float s0 = Ri[c], s1 = 0.f;
#pragma unroll
                    for (int t = 0; t < TB / 4; ++t) {
                        const float4 lv = Lc4[t];
                        s0 = fmaf(-g[4 * t], lv.x, s0);
                        s1 = fmaf(-g[4 * t + 1], lv.y, s1);
                        s0 = fmaf(-g[4 * t + 2], lv.z, s0);
                        s1 = fmaf(-g[4 * t + 3], lv.w, s1);
                    }
                    Ri[c] = s0 + s1;
                }
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < kTcBM * m; e += blockDim.x) {
        const int l = e / kTcBM, i = e % kTcBM;
        const int64_t gr = row0 + i;
        if (gr < N) F[(int64_t)(k + l) * ldf + gr] = Rs[i * (BN + 1) + l];
    }

    // ---- rho update and per-64-row tile statistics (threads 0..127 = rows) ----
    double rnew = 0.0, rmax = -1.0;
    int64_t ridx = LLONG_MAX;
    if (tid < kTcBM) {
        const int64_t gr = row0 + tid;
        const float* Ri = Rs + tid * (BN + 1);
        float nrm = 0.f;
        for (int l = 0; l < m; ++l) nrm = fmaf(Ri[l], Ri[l], nrm);
        if (gr < N) {
            rnew = fmax(rho[gr] - (double)nrm, 0.0);
            rho[gr] = rnew;
            rmax = rnew;
            ridx = gr;
        }
    }
    double sum = warp_sum(rnew);
    warp_argmax(rmax, ridx);
    if (lane == 0) {
        red[wid] = sum;
        redm[wid] = rmax;
        redi[wid] = ridx;
    }
    __syncthreads();
    if (tid < 2) {
        const int64_t t = 2 * (int64_t)blockIdx.x + tid;
        if (t * kBM < N) {
            double ts = red[2 * tid] + red[2 * tid + 1];
            double tm = redm[2 * tid];
            int64_t ti = redi[2 * tid];
            argmax_merge(tm, ti, redm[2 * tid + 1], redi[2 * tid + 1]);
            w.tile_sum[t] = ts;
            w.tile_max[t] = tm;
            w.tile_idx[t] = ti;
        }
    }
}

template <int BN>
static cudaError_t launch_bn(const FactorWs& w, const PanelWs& p, const float* X, float* F, int64_t ldf, double* rho,
                             int64_t N, int d, int b, double inv_eps, int r, cudaStream_t s) {
    const int nch = tc_chunks(d, r);
    k_panel<BN><<<nch, 256, 0, s>>>(w, p, d, b);
    k_lprep<BN><<<(BN * BN + 255) / 256, 256, 0, s>>>(w, p, b);
    const size_t smem = 2 * (2 * kTcBM * 128 + 2 * BN * 128) + BN * BN * 4 + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_engine_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((N + kTcBM - 1) / kTcBM);
    k_engine_tc<BN><<<grid, 256, smem, s>>>(w, p, X, F, ldf, rho, N, d, (float)inv_eps);
    return cudaGetLastError();
}

cudaError_t launch_engine_tc(const FactorWs& w, const PanelWs& p, const float* X, float* F, int64_t ldf, double* rho,
                             int64_t N, int d, int b, double inv_eps, int r, cudaStream_t s) {
    if (b <= 32) return launch_bn<32>(w, p, X, F, ldf, rho, N, d, b, inv_eps, r, s);
    if (b <= 64) return launch_bn<64>(w, p, X, F, ldf, rho, N, d, b, inv_eps, r, s);
    return launch_bn<128>(w, p, X, F, ldf, rho, N, d, b, inv_eps, r, s);
}

}  // namespace kevd
