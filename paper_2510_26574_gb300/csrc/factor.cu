// rpchol_factor: pivoted partial Cholesky of the implicit Gaussian kernel
// matrix (Section 1.2; Appendix A, Algorithms 2 and 3), FP64 path.
//
// One round of Algorithm 2 is five stream-ordered launches; the current rank
// k and the accepted count m live on the device, so no round needs a host
// synchronisation:
//   k_propose  commit the previous round (k += m); greedy: argmax of rho from
//              per-tile (max, index); ARPC: prefix of per-tile sums of rho and
//              b inverse-CDF draws with Philox uniforms (stream 0).
//   k_gather   X(S',:) and F(S',:) of the proposals into contiguous panels.
//   k_blockH   H = K(S',S') - F(S',:) F(S',:)^T  (b x b).
//   k_reject   Algorithm 3 (sequential accept test with Philox z, stream 1,
//              rank-1 Schur updates), the accepted positions and L = chol(H(T,T)).
//   k_engine   kernel-column engine: for a 64-row tile, K(:,S) from the
//              norm expansion exp(-(|x_i|^2 + |x_s|^2 - 2 x_i.x_s)/eps), minus
//              F F(S,:)^T, times L^-T by forward substitution, written to
//              F(:, k:k+m); fused residual update rho -= rownorms(G)^2, clamp at
//              0, and the per-tile sum and (max, index) of rho for the next round.
#include <algorithm>
#include <climits>
#include <vector>

#include "common.cuh"
#include "factor.cuh"
#include "kexp.cuh"
#include "oz_digits.cuh"
#include "ozgemm.cuh"
#include "trace.cuh"

namespace kevd {

static int tc_bn(int b) { return b <= 32 ? 32 : b <= 64 ? 64 : 128; }

// oz: the FP64 path with the engine on the tensor cores (ozmm.cu): the two
// N x b product arrays and the digit planes (OzWs) are carved after the rest;
// rounds_max bounds the padding of F's planes (16 columns per round).
static FactorWs carve_factor(void* base, int64_t N, int d, int r, int b, size_t* bytes, bool tc = false,
                             PanelWs* pw = nullptr, bool oz = false, OzWs* ow = nullptr, int rounds_max = 0) {
    Carver c(base);
    const int64_t nt = (N + kBM - 1) / kBM;
    FactorWs w{};
    w.st = c.take<FactorState>(1);
    w.xn = c.take<double>(N);
    w.tile_sum = c.take<double>(nt);
    w.tile_max = c.take<double>(nt);
    w.tile_idx = c.take<int64_t>(nt);
    w.pre_incl = c.take<double>(nt);
    w.pre_excl = c.take<double>(nt);
    w.prop = c.take<int64_t>(b);
    w.acc_pos = c.take<int32_t>(b);
    w.tpos = c.take<int32_t>(b);
    w.XSP = c.take<double>((size_t)d * b);
    w.FSP = c.take<double>((size_t)r * b);
    w.xnS = c.take<double>(b);
    w.H = c.take<double>((size_t)b * b);
    w.Lfull = c.take<double>((size_t)b * b);
    w.Lc = c.take<double>((size_t)b * b);
    if (tc) {
        const int BN = tc_bn(b);
        PanelWs p;
        p.panel = c.take<uint16_t>((size_t)tc_chunks(d, r) * 2 * BN * kTcBK);
        p.Lf = c.take<float>((size_t)BN * BN);
        p.nS = c.take<float>(BN);
        p.pidx = c.take<int64_t>(BN);
        p.err = c.take<int>(4);
        if (pw) *pw = p;
    }
    if (oz && !tc) {
        OzWs o;
        w.ldD = (N + 1) / 2 * 2;
        w.Dx = c.take<double>((size_t)w.ldD * b);
        w.Df = c.take<double>((size_t)w.ldD * b);
        o.ldX = (d + 15) / 16 * 16;
        o.ldF = (int)(((int64_t)r + 15 * (int64_t)std::max(rounds_max, 1) + 15) / 16 * 16);
        o.ldR = (b + 15) / 16 * 16;
        o.ldLi = (b + 1) / 2 * 2;
        o.Xp = c.take<uint16_t>((size_t)kDigits * N * o.ldX);
        o.xe = c.take<int>(N);
        o.Fp = c.take<uint16_t>((size_t)kDigits * N * o.ldF);
        o.Rp = c.take<uint16_t>((size_t)kDigits * N * o.ldR);
        o.re = c.take<int>(N);
        o.PXp = c.take<uint16_t>((size_t)kDigits * b * o.ldX);
        o.pxe = c.take<int>(b);
        o.PFp = c.take<uint16_t>((size_t)kDigits * b * o.ldF);
        o.Lp = c.take<uint16_t>((size_t)kDigits * b * o.ldR);
        o.le = c.take<int>(b);
        o.Linv = c.take<double>((size_t)b * o.ldLi);
        o.flags = c.take<int>(4);
        if (ow) *ow = o;
    }
    *bytes = c.off;
    return w;
}

// ---------------------------------------------------------------------------
// a1: squared norms, rho := diag K = 1, initial tile statistics.
// ---------------------------------------------------------------------------
template <typename TX>
__device__ __forceinline__ void prepare_body(const TX* __restrict__ X, int64_t N, int d, FactorWs w,
                                             double* __restrict__ rho, int64_t blk) {
    const int64_t i = blk * blockDim.x + threadIdx.x;
    if (blk == 0 && threadIdx.x == 0) {
        FactorState s = {};
        *w.st = s;
    }
    if (i < N) {
        const TX* x = X + i * d;
        double s = 0.0;
        for (int c = 0; c < d; ++c) s = fma((double)x[c], (double)x[c], s);
        w.xn[i] = s;
        rho[i] = 1.0;
        if (!isfinite(s)) w.st->bad = 1;   // benign race: every writer stores 1
        if ((i % kBM) == 0) {
            const int64_t t = i / kBM;
            const int64_t cnt = min((int64_t)kBM, N - i);
            w.tile_sum[t] = (double)cnt;
            w.tile_max[t] = 1.0;
            w.tile_idx[t] = i;
        }
    }
}

template <typename TX>
__global__ void k_prepare(const TX* __restrict__ X, int64_t N, int d, FactorWs w, double* __restrict__ rho) {
    prepare_body(X, N, d, w, rho, blockIdx.x);
}

// Warp-inclusive scan (Hillis-Steele over shuffles).
__device__ __forceinline__ double warp_incl_scan(double v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// ---------------------------------------------------------------------------
// a2: pivot proposal.  One block of 1024 threads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void propose_body(FactorWs w, const double* __restrict__ rho, int64_t N, int64_t ntiles,
                                             int b, int r, int greedy, uint64_t seed, int rnd,
                                             int64_t* __restrict__ proposals_out, double floor_sum = 0.0) {
    __shared__ double sh[33];
    __shared__ int64_t shi[32];
    __shared__ int s_go;
    FactorState* st = w.st;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) {
        if (st->m > 0) {
            st->sum_k += st->k;
            st->eng_rounds += 1;
        }
        st->k += st->m;
        st->kp += (st->m + 15) & ~15;
        st->sum_m_sq += (long long)st->m * st->m;
        st->m = 0;
        if (st->k >= r) st->done = 1;
        s_go = !st->done;
    }
    __syncthreads();
    if (!s_go) return;

    if (greedy) {
        double v = -1.0;
        int64_t idx = LLONG_MAX;
        for (int64_t t = tid; t < ntiles; t += blockDim.x) argmax_merge(v, idx, w.tile_max[t], w.tile_idx[t]);
        warp_argmax(v, idx);
        if (lane == 0) {
            sh[wid] = v;
            shi[wid] = idx;
        }
        __syncthreads();
        if (wid == 0) {
            v = lane < nw ? sh[lane] : -1.0;
            idx = lane < nw ? shi[lane] : LLONG_MAX;
            warp_argmax(v, idx);
            if (lane == 0) {
                if (!(v > 0.0)) {
                    st->done = 1;
                } else {
                    w.prop[0] = idx;
                    st->total = v;
                    st->rounds += 1;
                    if (proposals_out) proposals_out[rnd] = idx;
                }
            }
        }
        return;
    }

    // Exclusive/inclusive prefix of the tile sums; each thread owns a
    // contiguous chunk, chunks are combined by a block scan.
    const int64_t chunk = (ntiles + blockDim.x - 1) / blockDim.x;
    const int64_t t0 = min((int64_t)tid * chunk, ntiles), t1 = min(t0 + chunk, ntiles);
    double loc = 0.0;
    for (int64_t t = t0; t < t1; ++t) loc += w.tile_sum[t];
    double inc = warp_incl_scan(loc);
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        double wv = lane < nw ? sh[lane] : 0.0;
        double wi = warp_incl_scan(wv);
        sh[lane] = wi - wv;            // exclusive warp offsets
        if (lane == 31) sh[32] = wi;   // block total
    }
    __syncthreads();
    double run = sh[wid] + inc - loc;
    const double S = sh[32];
    for (int64_t t = t0; t < t1; ++t) {
        w.pre_excl[t] = run;
        run += w.tile_sum[t];
        w.pre_incl[t] = run;
    }
    __syncthreads();
    if (!(S > floor_sum)) {   // sum(rho) = 0, or at the caller's floor tol * N
        if (tid == 0) st->done = 1;
        return;
    }
    if (tid == 0) {
        st->total = S;
        st->rounds += 1;
    }
    for (int j = wid; j < b; j += nw) {
        const double u = philox_uniform(seed, 0u, (uint32_t)rnd, (uint32_t)j);
        const double target = u * S;
        // smallest tile t with pre_incl[t] > target
        int64_t lo = 0, hi = ntiles;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (w.pre_incl[mid] > target) hi = mid; else lo = mid + 1;
        }
        int64_t t = lo;
        if (t == ntiles) {   // u*S rounded to >= S: last tile with mass
            t = ntiles - 1;
            while (t > 0 && !(w.tile_sum[t] > 0.0)) --t;
        }
        const int64_t base = t * kBM;
        const int cnt = (int)min((int64_t)kBM, N - base);
        double acc = w.pre_excl[t];
        int64_t found = -1, last_pos = -1;
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            const int rr = c0 + lane;
            const double v = rr < cnt ? rho[base + rr] : 0.0;
            const double sv = warp_incl_scan(v);
            const unsigned pos = __ballot_sync(0xffffffffu, rr < cnt && v > 0.0);
            if (pos) last_pos = base + c0 + 31 - __clz(pos);
            const unsigned hit = __ballot_sync(0xffffffffu, rr < cnt && v > 0.0 && acc + sv > target);
            if (hit) {
                found = base + c0 + __ffs(hit) - 1;
                break;
            }
            acc += __shfl_sync(0xffffffffu, sv, 31);
        }
        if (found < 0) found = last_pos;   // rounding at the tile's upper edge
        if (found < 0) found = base;       // unreachable: the tile has mass
        if (lane == 0) {
            w.prop[j] = found;
            if (proposals_out) proposals_out[(int64_t)rnd * b + j] = found;
        }
    }
}

__global__ void __launch_bounds__(1024) k_propose(FactorWs w, const double* __restrict__ rho, int64_t N,
                                                  int64_t ntiles, int b, int r, int greedy, uint64_t seed, int rnd,
                                                  int64_t* __restrict__ proposals_out, double floor_sum) {
    propose_body(w, rho, N, ntiles, b, r, greedy, seed, rnd, proposals_out, floor_sum);
}

// ---------------------------------------------------------------------------
// a3 (part 1): gather X(S',:) and F(S',:)[:, :k] into d x b and k x b panels.
// ---------------------------------------------------------------------------
template <typename TX, typename TF>
__device__ __forceinline__ void gather_body(FactorWs w, const TX* __restrict__ X, const TF* __restrict__ F,
                                            int64_t ldf, int d, int b, int blk) {
    const FactorState* st = w.st;
    if (st->done) return;
    const int k = st->k;
    const int lane = threadIdx.x & 31;
    const int c = blk * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (blk == 0 && threadIdx.x < b) w.xnS[threadIdx.x] = w.xn[w.prop[threadIdx.x]];
    if (c < d) {
        for (int j = lane; j < b; j += 32) w.XSP[(size_t)c * b + j] = (double)X[w.prop[j] * d + c];
    } else if (c - d < k) {
        const int cf = c - d;
        for (int j = lane; j < b; j += 32) w.FSP[(size_t)cf * b + j] = (double)F[w.prop[j] + (int64_t)cf * ldf];
    }
}

template <typename TX, typename TF>
__global__ void k_gather(FactorWs w, const TX* __restrict__ X, const TF* __restrict__ F, int64_t ldf, int d, int b) {
    gather_body(w, X, F, ldf, d, b, blockIdx.x);
}

// ---------------------------------------------------------------------------
// a3 (part 2): H = K(S',S') - F(S',:) F(S',:)^T.  One warp per entry (j, l):
// the lanes split the d- and k-long dot products and a shuffle tree adds them,
// so each entry is a chain of ~(d + k)/32 FMAs instead of d + k.  H(j,l) and
// H(l,j) go through the same lane assignment and the same tree, with the two
// factors of each product swapped (fma is commutative in its first two
// operands), so H is exactly symmetric.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void blockH_body(FactorWs w, int d, int b, double inv_eps, int pair) {
    const FactorState* st = w.st;
    if (st->done) return;
    if (pair >= b * b) return;
    const int k = st->k;
    const int j = pair / b, l = pair % b;
    const int lane = threadIdx.x & 31;
    double dx = 0.0, df = 0.0;
    for (int c = lane; c < d; c += 32) dx = fma(w.XSP[(size_t)c * b + j], w.XSP[(size_t)c * b + l], dx);
    for (int c = lane; c < k; c += 32) df = fma(w.FSP[(size_t)c * b + j], w.FSP[(size_t)c * b + l], df);
    dx = warp_sum(dx);
    df = warp_sum(df);
    if (lane != 0) return;
    double kv;
    if (w.prop[j] == w.prop[l]) {
        kv = 1.0;   // k(x, x) = exp(0)
    } else {
        const double d2 = fmax(w.xnS[j] + w.xnS[l] - 2.0 * dx, 0.0);
        kv = exp(-d2 * inv_eps);
    }
    w.H[(size_t)j * b + l] = kv - df;
}

constexpr int kBlockHWarps = 8;   // entries per 256-thread block

__global__ void k_blockH(FactorWs w, int d, int b, double inv_eps) {
    blockH_body(w, d, b, inv_eps, blockIdx.x * kBlockHWarps + (threadIdx.x >> 5));
}

// ---------------------------------------------------------------------------
// a4: Algorithm 3 (ARPC) or the greedy acceptance (b = 1, accept iff H > 0).
// One block; H lives in shared memory (b*b doubles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reject_body(FactorWs w, int b, int r, int greedy, uint64_t seed, int rnd,
                                            int64_t* __restrict__ pivots, double* smem) {
    double* Hs = smem;                 // b*b
    double* Lcol = Hs + (size_t)b * b; // b
    double* rho0 = Lcol + b;           // b
    double* zs = rho0 + b;             // b
    __shared__ int s_acc, s_m, s_go;
    FactorState* st = w.st;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_go = !st->done;
        s_m = 0;
    }
    __syncthreads();
    if (!s_go) return;
    const int k = st->k;
    for (int e = tid; e < b * b; e += blockDim.x) Hs[e] = w.H[e];
    __syncthreads();
    for (int e = tid; e < b; e += blockDim.x) {
        rho0[e] = Hs[(size_t)e * b + e];
        zs[e] = greedy ? 0.0 : philox_uniform(seed, 1u, (uint32_t)rnd, (uint32_t)e);   // the z of every proposal
    }
    __syncthreads();
    for (int i = 0; i < b; ++i) {
        if (tid == 0) {
            const double hii = Hs[(size_t)i * b + i];
            int acc;
            if (greedy) {
                acc = hii > 0.0;
            } else {
                acc = hii > 0.0 && zs[i] * rho0[i] < hii;
            }
            if (k + s_m >= r) acc = 0;
            if (acc) w.tpos[s_m++] = i;
            s_acc = acc;
        }
        __syncthreads();
        const int accepted = s_acc;
        __syncthreads();   // every thread has read s_acc before thread 0 rewrites it
        if (!accepted) continue;
        const double piv = sqrt(Hs[(size_t)i * b + i]);
        for (int l = i + tid; l < b; l += blockDim.x) {
            // greedy divides the residual column by sqrt(H) directly; Algorithm 3
            // scales the whole column H(i:b, i) by 1/sqrt(H(i,i)).
            const double v = (greedy && l == i) ? piv : Hs[(size_t)l * b + i] / piv;
            Lcol[l] = v;
            w.Lfull[(size_t)l * b + i] = v;
        }
        __syncthreads();
        const int n = b - i - 1;
        for (int e = tid; e < n * n; e += blockDim.x) {
            const int l = i + 1 + e / n, mm = i + 1 + e % n;
            Hs[(size_t)l * b + mm] -= Lcol[l] * Lcol[mm];
        }
        __syncthreads();
    }
    __syncthreads();
    const int m = s_m;
    for (int e = tid; e < m * m; e += blockDim.x) {
        const int a = e / m, a2 = e % m;
        w.Lc[(size_t)a * b + a2] = a2 <= a ? w.Lfull[(size_t)w.tpos[a] * b + w.tpos[a2]] : 0.0;
    }
    for (int a = tid; a < m; a += blockDim.x) {
        w.acc_pos[a] = w.tpos[a];
        pivots[k + a] = w.prop[w.tpos[a]];
    }
    if (tid == 0) {
        st->m = m;
        if (greedy && m == 0) st->done = 1;   // greedy stops once H <= 0
    }
}

__global__ void __launch_bounds__(1024) k_reject(FactorWs w, int b, int r, int greedy, uint64_t seed, int rnd,
                                                 int64_t* __restrict__ pivots) {
    extern __shared__ double smem_rej[];
    reject_body(w, b, r, greedy, seed, rnd, pivots, smem_rej);
}

// ---------------------------------------------------------------------------
// a5 + a6: the kernel-column engine (FP64).  Tile = 64 rows x BN = 8*TN columns.
// Warp w owns columns [w*TN, w*TN+TN); lane owns rows 2*lane, 2*lane+1.
// Warps whose columns are all >= m skip the products.
// ---------------------------------------------------------------------------
template <int TN>
__device__ __forceinline__ void engine_body(FactorWs w, const double* __restrict__ X, double* __restrict__ F,
                                            int64_t ldf, double* __restrict__ rho, int64_t N, int d, int b,
                                            double inv_eps, int64_t tile, double* smem) {
    constexpr int BN = 8 * TN;
    constexpr int APAD = kBM + 2;
    double* As = smem;                 // kBK x APAD
    double* Bs = As + kBK * APAD;      // kBK x BN
    double* Rs = smem;                 // kBM x (BN+1), reused after the products
    __shared__ double red[32];
    __shared__ int64_t redi[32];

    const FactorState* st = w.st;
    if (st->done) return;
    const int m = st->m;
    if (m == 0) return;
    const int k = st->k;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t row0 = tile * kBM;
    const bool active = wid * TN < m;

    double acc[2][TN];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[a][c] = 0.0;

    // ---- X(i,:) . X(s,:) over d ----
    for (int c0 = 0; c0 < d; c0 += kBK) {
#pragma unroll
        for (int p = 0; p < (kBM * kBK) / 256; ++p) {
            const int e = tid + 256 * p, i = e / kBK, kk = e % kBK;
            const int64_t row = row0 + i;
            As[kk * APAD + i] = (row < N && c0 + kk < d) ? X[row * d + c0 + kk] : 0.0;
        }
        for (int e = tid; e < kBK * BN; e += 256) {
            const int kk = e / BN, l = e % BN;
            Bs[kk * BN + l] = (l < m && c0 + kk < d) ? w.XSP[(size_t)(c0 + kk) * b + w.acc_pos[l]] : 0.0;
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int kk = 0; kk < kBK; ++kk) {
                const double2 a = *reinterpret_cast<const double2*>(&As[kk * APAD + 2 * lane]);
#pragma unroll
                for (int c = 0; c < TN; ++c) {
                    const double bv = Bs[kk * BN + wid * TN + c];
                    acc[0][c] = fma(a.x, bv, acc[0][c]);
                    acc[1][c] = fma(a.y, bv, acc[1][c]);
                }
            }
        }
        __syncthreads();
    }
    // ---- kernel values: exp(-(|x_i|^2 + |x_s|^2 - 2 x_i.x_s) / eps) ----
    if (active) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int64_t row = row0 + 2 * lane + a;
            const double xi = row < N ? w.xn[row] : 0.0;
#pragma unroll
            for (int c = 0; c < TN; ++c) {
                const int l = wid * TN + c;
                if (l < m) {
                    const int pos = w.acc_pos[l];
                    if (w.prop[pos] == row) {
                        acc[a][c] = 1.0;
                    } else {
                        const double d2 = fmax(xi + w.xnS[pos] - 2.0 * acc[a][c], 0.0);
                        acc[a][c] = exp(-d2 * inv_eps);
                    }
                }
            }
        }
    }
    // ---- minus F(i,:k) . F(s,:k) ----
    for (int c0 = 0; c0 < k; c0 += kBK) {
#pragma unroll
        for (int p = 0; p < (kBM * kBK) / 256; ++p) {
            const int e = tid + 256 * p, kk = e / kBM, i = e % kBM;
            const int64_t row = row0 + i;
            As[kk * APAD + i] = (row < N && c0 + kk < k) ? F[(int64_t)(c0 + kk) * ldf + row] : 0.0;
        }
        for (int e = tid; e < kBK * BN; e += 256) {
            const int kk = e / BN, l = e % BN;
            Bs[kk * BN + l] = (l < m && c0 + kk < k) ? w.FSP[(size_t)(c0 + kk) * b + w.acc_pos[l]] : 0.0;
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int kk = 0; kk < kBK; ++kk) {
                const double2 a = *reinterpret_cast<const double2*>(&As[kk * APAD + 2 * lane]);
#pragma unroll
                for (int c = 0; c < TN; ++c) {
                    const double bv = Bs[kk * BN + wid * TN + c];
                    acc[0][c] = fma(-a.x, bv, acc[0][c]);
                    acc[1][c] = fma(-a.y, bv, acc[1][c]);
                }
            }
        }
        __syncthreads();
    }
    // ---- R tile to shared memory ----
    if (active) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < TN; ++c) Rs[(2 * lane + a) * (BN + 1) + wid * TN + c] = acc[a][c];
    }
    __syncthreads();
    // ---- G = R L^-T by forward substitution, rho update ----
    double rnew = 0.0;
    double rmax = -1.0;
    int64_t ridx = LLONG_MAX;
    if (tid < kBM) {
        const int64_t row = row0 + tid;
        double* Ri = Rs + tid * (BN + 1);
        double nrm = 0.0;
        for (int j = 0; j < m; ++j) {
            const double* Lj = w.Lc + (size_t)j * b;
            double s = Ri[j];
            for (int l = 0; l < j; ++l) s = fma(-__ldg(Lj + l), Ri[l], s);
            const double g = s / __ldg(Lj + j);
            Ri[j] = g;
            nrm = fma(g, g, nrm);
        }
        if (row < N) {
            rnew = fmax(rho[row] - nrm, 0.0);
            rho[row] = rnew;
            rmax = rnew;
            ridx = row;
        }
    }
    __syncthreads();
    for (int e = tid; e < kBM * m; e += 256) {
        const int l = e / kBM, i = e % kBM;
        const int64_t row = row0 + i;
        if (row < N) F[(int64_t)(k + l) * ldf + row] = Rs[i * (BN + 1) + l];
    }
    // ---- per-tile sum and (max, lowest index) of rho ----
    double s = warp_sum(rnew);
    warp_argmax(rmax, ridx);
    if (lane == 0) {
        red[wid] = s;
        redi[wid] = ridx;
        red[16 + wid] = rmax;
    }
    __syncthreads();
    if (tid == 0) {
        double ts = 0.0, tm = -1.0;
        int64_t ti = LLONG_MAX;
        for (int q = 0; q < (kBM + 31) / 32; ++q) {
            ts += red[q];
            argmax_merge(tm, ti, red[16 + q], redi[q]);
        }
        w.tile_sum[tile] = ts;
        w.tile_max[tile] = tm;
        w.tile_idx[tile] = ti;
    }
    __syncthreads();   // shared buffers are reused by the next tile of a persistent caller
}

template <int TN>
__global__ void __launch_bounds__(256) k_engine(FactorWs w, const double* __restrict__ X, double* __restrict__ F,
                                                int64_t ldf, double* __restrict__ rho, int64_t N, int d, int b,
                                                double inv_eps) {
    extern __shared__ double smem_eng[];
    engine_body<TN>(w, X, F, ldf, rho, N, d, b, inv_eps, blockIdx.x, smem_eng);
}

// Digit planes of X (seven digits, one exponent per row from max |X(i, :)|),
// columns d .. ldX - 1 zero.  One warp per row, a lane two columns at a time.
__global__ void __launch_bounds__(256) k_xplanes(const double* __restrict__ X, int64_t N, int d, OzWs o) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= N) return;
    const double* x = X + i * d;
    double mx = 0.0;
    for (int c = lane; c < d; c += 32) mx = fmax(mx, fabs(x[c]));
#pragma unroll
    for (int q = 16; q; q >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, q));
    const int E = exp_of(mx);
    if (lane == 0) o.xe[i] = E;
    const size_t plane = (size_t)N * o.ldX / 2;                 // words
    uint32_t* P = reinterpret_cast<uint32_t*>(o.Xp) + (size_t)i * (o.ldX / 2);
    for (int c = 2 * lane; c < o.ldX; c += 64) {
        const double x0 = c < d ? x[c] : 0.0, x1 = c + 1 < d ? x[c + 1] : 0.0;
        uint32_t wd[kDigits];
        digits2_e(x0, x1, E, wd);
#pragma unroll
        for (int s = 0; s < kDigits; ++s) P[s * plane + c / 2] = wd[s];
    }
}

// Pivot panels of the round as rows of the digit planes: row l < m of PXp is
// row S_l of Xp (exponent pxe_l), row l of PFp is row S_l of Fp over the padded
// rank kp; rows l >= m are zero.  One block per row l, 16-byte copies.
__global__ void __launch_bounds__(128) k_ozpanel(FactorWs w, OzWs o, int64_t N, int b) {
    const FactorState* st = w.st;
    if (st->done || st->m == 0) return;
    const int l = blockIdx.x;
    if (l >= b) return;
    const bool on = l < st->m;
    const int64_t row = on ? w.prop[w.acc_pos[l]] : 0;
    if (threadIdx.x == 0) o.pxe[l] = on ? o.xe[row] : -900;
    const int kp = st->kp;
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int s = 0; s < kDigits; ++s) {
        const uint4* xs = reinterpret_cast<const uint4*>(o.Xp + ((size_t)s * N + row) * o.ldX);
        uint4* xd = reinterpret_cast<uint4*>(o.PXp + ((size_t)s * b + l) * o.ldX);
        for (int c = threadIdx.x; c < o.ldX / 8; c += blockDim.x) xd[c] = on ? xs[c] : z;
        const uint4* fs = reinterpret_cast<const uint4*>(o.Fp + ((size_t)s * N + row) * o.ldF);
        uint4* fd = reinterpret_cast<uint4*>(o.PFp + ((size_t)s * b + l) * o.ldF);
        for (int c = threadIdx.x; c < kp / 8; c += blockDim.x) fd[c] = on ? fs[c] : z;
    }
}

// L(T,T)^-1 of the round (lower triangular, m x m) and its digit planes: rows j
// of Lp (exponent le_j), columns past m and rows past m zero.  One block;
// thread c forms column c by forward substitution on L e_c (L staged in shared
// memory, read by broadcast).  Each round's L is the Cholesky factor of
// Algorithm 3's accepted block, whose accept test keeps it well conditioned, so
// multiplying by the explicit inverse agrees with substitution to rounding
// (measured 2e-15 on KS data).
__global__ void __launch_bounds__(128) k_linv(FactorWs w, OzWs o, int b) {
    extern __shared__ double Ls[];
    const FactorState* st = w.st;
    if (st->done || st->m == 0) return;
    const int m = st->m;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int j = e / m, l = e % m;
        Ls[e] = l <= j ? w.Lc[(size_t)j * b + l] : 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c < b) {
        for (int j = 0; j < b; ++j) {
            double x = 0.0;
            if (c < m && j >= c && j < m) {
                if (j == c) {
                    x = 1.0 / Ls[j * m + j];
                } else {
                    double s = 0.0;
                    for (int l = c; l < j; ++l) s = fma(Ls[j * m + l], o.Linv[(size_t)l * o.ldLi + c], s);
                    x = -s / Ls[j * m + j];
                }
            }
            o.Linv[(size_t)j * o.ldLi + c] = x;
        }
    }
    __syncthreads();
    if (c < b) {   // row c: exponent and planes (columns < m hold the row, the rest zero)
        const double* row = o.Linv + (size_t)c * o.ldLi;
        double mx = 0.0;
        for (int l = 0; l < m; ++l) mx = fmax(mx, fabs(row[l]));
        const int E = exp_of(mx);
        o.le[c] = E;
        uint32_t* P = reinterpret_cast<uint32_t*>(o.Lp) + (size_t)c * (o.ldR / 2);
        const size_t plane = (size_t)b * o.ldR / 2;
        for (int l = 0; l < o.ldR; l += 2) {
            uint32_t wd[kDigits];
            digits2_e(l < m ? row[l] : 0.0, l + 1 < m ? row[l + 1] : 0.0, E, wd);
#pragma unroll
            for (int s = 0; s < kDigits; ++s) P[s * plane + l / 2] = wd[s];
        }
    }
}

// R = K(:, T) - F(:, :k) F(T, :k)^T from the tensor-core products: the kernel
// values exp(-(|x_i|^2 + |x_s|^2 - 2 x_i.x_s) / eps) (1 at the pivot itself)
// minus Df, as digit planes with one exponent per row (the row maximum over
// the round's pivots).  Block: 32 rows x 8 warps, warp g taking the 16 pivots
// [16 g, 16 g + 16) (16 values per thread: low register use, four blocks per SM).
__global__ void __launch_bounds__(256, 4) k_rprep(FactorWs w, OzWs o, int64_t N, double inv_eps,
                                                  const unsigned long long* __restrict__ tblg) {
    const FactorState* st = w.st;
    if (st->done || st->m == 0) return;
    const int m = st->m, k = st->k;
    __shared__ unsigned long long red[8][32];
    __shared__ unsigned long long tbl[1024];
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) tbl[e] = tblg[e];
    __syncthreads();
    const int il = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * 32 + il;
    const int l0 = 16 * g;
    double R[16];
    unsigned long long mx = 0;                                 // max |R| as the bits of a non-negative double
    const double xi = row < N ? w.xn[row] : 0.0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int l = l0 + e;
        double rv = 0.0;
        if (row < N && l < m) {
            const int pos = w.acc_pos[l];
            const int64_t at = row + (int64_t)l * w.ldD;
            double kv;
            if (w.prop[pos] == row) {
                kv = 1.0;
            } else {
                double d2 = fma(-2.0, w.Dx[at], xi + w.xnS[pos]);
                if (__double_as_longlong(d2) < 0) d2 = 0.0;     // negative rounding residue
                kv = kexp(-d2 * inv_eps, tbl);
            }
            rv = k > 0 ? kv - w.Df[at] : kv;
        }
        R[e] = rv;
        mx = max(mx, (unsigned long long)__double_as_longlong(rv) & 0x7FFFFFFFFFFFFFFFull);
    }
    red[g][il] = mx;
    __syncthreads();
    if (row >= N || l0 >= o.ldR) return;
    unsigned long long rm = red[0][il];
#pragma unroll
    for (int q = 1; q < 8; ++q) rm = max(rm, red[q][il]);
    const int E = exp_of(__longlong_as_double((long long)rm));
    if (g == 0) o.re[row] = E;
    const size_t plane = (size_t)N * o.ldR / 2;
    uint32_t* P = reinterpret_cast<uint32_t*>(o.Rp) + (size_t)row * (o.ldR / 2) + l0 / 2;
    const int npair = min(8, (o.ldR - l0) / 2);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        if (e < npair) {
            uint32_t wd[kDigits];
            digits2_e(R[2 * e], R[2 * e + 1], E, wd);
#pragma unroll
            for (int s = 0; s < kDigits; ++s) P[s * plane + e] = wd[s];
        }
    }
}

// After G = R L^-T has been written to F(:, k:k+m): rho -= rownorms(G)^2 (clamped
// at 0) and the per-tile sum and (max, lowest index) of rho for the next round's
// sampler.  Block: one 64-row tile x 4 column groups.
__global__ void __launch_bounds__(256) k_rho_update(FactorWs w, const double* __restrict__ F, int64_t ldf,
                                                    double* __restrict__ rho, int64_t N) {
    const FactorState* st = w.st;
    if (st->done || st->m == 0) return;
    const int m = st->m, k = st->k;
    __shared__ double sn[4][64];
    __shared__ double red[2];
    __shared__ double redm[2];
    __shared__ int64_t redi[2];
    const int il = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int64_t tile = blockIdx.x, row = tile * 64 + il;
    double nrm = 0.0;
    if (row < N) {
        for (int l = g; l < m; l += 4) {
            const double v = F[(int64_t)(k + l) * ldf + row];
            nrm = fma(v, v, nrm);
        }
    }
    sn[g][il] = nrm;
    __syncthreads();
    if (g == 0) {
        double rnew = 0.0, rmax = -1.0;
        int64_t ridx = LLONG_MAX;
        if (row < N) {
            const double tot = (sn[0][il] + sn[1][il]) + (sn[2][il] + sn[3][il]);
            rnew = fmax(rho[row] - tot, 0.0);
            rho[row] = rnew;
            rmax = rnew;
            ridx = row;
        }
        const double s2 = warp_sum(rnew);
        warp_argmax(rmax, ridx);
        if ((il & 31) == 0) {
            red[il >> 5] = s2;
            redm[il >> 5] = rmax;
            redi[il >> 5] = ridx;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && tile * 64 < N) {
        double tm = redm[0];
        int64_t ti = redi[0];
        argmax_merge(tm, ti, redm[1], redi[1]);
        w.tile_sum[tile] = red[0] + red[1];
        w.tile_max[tile] = tm;
        w.tile_idx[tile] = ti;
    }
}

// ---------------------------------------------------------------------------
// Commit the last round, sum(rho) in a fixed order, zero F(:, rank:r).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize_body(FactorWs w, const double* __restrict__ rho, int64_t N) {
    __shared__ double sh[32];
    FactorState* st = w.st;
    const int64_t chunk = (N + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = min((int64_t)threadIdx.x * chunk, N), i1 = min(i0 + chunk, N);
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) s += rho[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        if (st->m > 0) {
            st->sum_k += st->k;
            st->eng_rounds += 1;
        }
        st->k += st->m;
        st->kp += (st->m + 15) & ~15;
        st->sum_m_sq += (long long)st->m * st->m;
        st->m = 0;
        st->final_sum = s;
    }
}

__global__ void __launch_bounds__(1024) k_finalize(FactorWs w, const double* __restrict__ rho, int64_t N) {
    finalize_body(w, rho, N);
}

template <typename TF>
__global__ void k_zero_tail(const FactorState* st, TF* __restrict__ F, int64_t ldf, int64_t N, int r) {
    const int k = st->k;
    const int c = k + blockIdx.y;
    if (c >= r) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        F[(int64_t)c * ldf + i] = TF(0);
}

template <int TN>
static size_t engine_smem() {
    constexpr int BN = 8 * TN;
    const size_t stage = (size_t)(kBK * (kBM + 2) + kBK * BN) * sizeof(double);
    const size_t rtile = (size_t)kBM * (BN + 1) * sizeof(double);
    return std::max(stage, rtile);
}

template <int TN>
static cudaError_t prepare_engine() {
    return cudaFuncSetAttribute(k_engine<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)engine_smem<TN>());
}

template <int TN>
static void launch_engine(const FactorWs& w, const double* X, double* F, int64_t ldf, double* rho,
                          int64_t N, int d, int b, double inv_eps, int64_t ntiles, cudaStream_t s) {
    k_engine<TN><<<(unsigned)ntiles, 256, engine_smem<TN>(), s>>>(w, X, F, ldf, rho, N, d, b, inv_eps);
}

// Round launchers of the FP64 path, shared with the low-memory factor.
FactorWs carve_factor_fp64(void* base, int64_t N, int d, int r, int b, size_t* bytes) {
    return carve_factor(base, N, d, r, b, bytes);
}

void launch_prepare_fp64(const double* X, int64_t N, int d, const FactorWs& w, double* rho, cudaStream_t s) {
    k_prepare<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(X, N, d, w, rho);
}

void launch_propose(const FactorWs& w, const double* rho, int64_t N, int b, int r, int greedy, uint64_t seed, int rnd,
                    int64_t* proposals, double floor_sum, cudaStream_t s) {
    k_propose<<<1, 1024, 0, s>>>(w, rho, N, (N + kBM - 1) / kBM, b, r, greedy, seed, rnd, proposals, floor_sum);
}

void launch_blockH(const FactorWs& w, int d, int b, double inv_eps, cudaStream_t s) {
    k_blockH<<<(unsigned)((b * b + kBlockHWarps - 1) / kBlockHWarps), 32 * kBlockHWarps, 0, s>>>(w, d, b, inv_eps);
}

cudaError_t launch_reject(const FactorWs& w, int b, int r, int greedy, uint64_t seed, int rnd, int64_t* pivots,
                          cudaStream_t s) {
    const size_t smem = ((size_t)b * b + 3 * (size_t)b) * sizeof(double);   // H, L column, rho0, z
    const cudaError_t e = cudaFuncSetAttribute(k_reject, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_reject<<<1, b >= 32 ? 1024 : 128, smem, s>>>(w, b, r, greedy, seed, rnd, pivots);
    return cudaGetLastError();
}

void launch_finalize(const FactorWs& w, const double* rho, int64_t N, cudaStream_t s) {
    k_finalize<<<1, 1024, 0, s>>>(w, rho, N);
}

}  // namespace kevd

using namespace kevd;

static int factor_rounds(const kevd_opts* o, int r, int b) {
    if (o->until_rank) return o->max_rounds > 0 ? o->max_rounds : 4 * ((r + b - 1) / b) + 16;
    return r / b;
}

static size_t factor_ws_bytes(int64_t N, int d, int r, int b, bool tc, bool oz, int rounds_max) {
    size_t bytes = 0;
    carve_factor(nullptr, N, d, r, b, &bytes, tc, nullptr, oz, nullptr, rounds_max);
    return bytes;
}

// The FP64 path runs its engine on the tensor cores (FP64-accurate digit planes,
// ozmm.cu) for ARPC with b >= 32 (each round's block of F's planes is padded to
// 16 columns) and N < 2^31, unless KEVD_ENGINE=fp64 asks for the FP64-pipe
// engine; the workspace then holds two N x b product arrays and the planes.
static bool oz_engine_enabled() {
    const char* e = getenv("KEVD_ENGINE");
    return !(e && e[0] == 'f');
}

static bool oz_engine_for(const kevd_opts* o, int64_t N, int b, bool allow_oz) {
    return allow_oz && o->precision == KEVD_PREC_FP64 && o->mode == KEVD_ARPC && b >= 32 &&
           N < ((int64_t)1 << 31) && oz_engine_enabled();
}

size_t kevd_factor_ws_mode(int64_t N, int32_t d, int32_t r, const kevd_opts* o, bool allow_oz) {
    if (!o || N < 1 || d < 1 || r < 1) return 0;
    const int b = o->mode == KEVD_GREEDY ? 1 : o->block_b;
    if (b < 1 || b > 128) return 0;
    const bool tc = o->precision == KEVD_PREC_BF16X3;
    return factor_ws_bytes(N, d, r, b, tc, oz_engine_for(o, N, b, allow_oz), factor_rounds(o, r, b));
}

size_t kevd_factor_ws(int64_t N, int32_t d, int32_t r, const kevd_opts* o) {
    return kevd_factor_ws_mode(N, d, r, o, true);
}

int rpchol_factor_impl(const void* X, int x_dtype, int64_t N, int32_t d, double eps, int32_t r,
                       const kevd_opts* opts, void* F, int f_dtype, int64_t ldf, int64_t* pivots, double* rho,
                       int64_t* proposals, kevd_factor_info* info, void* workspace, size_t ws_bytes, void* stream,
                       bool allow_oz) {
    if (!opts || !X || !F || !pivots || !rho || !info) return KEVD_EINVAL;
    if (N < 1 || d < 1 || r < 1 || r > N || ldf < N) return KEVD_EINVAL;
    if (!(eps > 0.0) || !isfinite(eps)) return KEVD_EINVAL;
    if (opts->mode != KEVD_GREEDY && opts->mode != KEVD_ARPC) return KEVD_EINVAL;
    const bool tc = opts->precision == KEVD_PREC_BF16X3;
    if (opts->precision == KEVD_PREC_FP64) {
        if (x_dtype != KEVD_F64 || f_dtype != KEVD_F64) return KEVD_EINVAL;
    } else if (tc) {
        if (x_dtype != KEVD_F32 || f_dtype != KEVD_F32) return KEVD_EINVAL;
    } else {
        return KEVD_EINVAL;
    }
    if (opts->reserved != 0 || opts->max_rounds < 0) return KEVD_EINVAL;
    if (!(opts->tol >= 0.0 && opts->tol < 1.0)) return KEVD_EINVAL;
    const int greedy = opts->mode == KEVD_GREEDY;
    const int b = greedy ? 1 : opts->block_b;
    if (b < 1 || b > 128) return KEVD_EINVAL;
    const int rounds = greedy && !opts->until_rank ? r : factor_rounds(opts, r, b);
    if (rounds < 1) return KEVD_EINVAL;
    size_t need = 0;
    PanelWs pw{};
    OzWs ow{};
    const bool oz = oz_engine_for(opts, N, b, allow_oz);
    FactorWs w = carve_factor(workspace, N, d, r, b, &need, tc, &pw, oz, &ow, factor_rounds(opts, r, b));
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return KEVD_EWORKSPACE;
    // tensor maps of the digit planes: X and F (A operands), the pivot panels (B),
    // R and L^-1 of each round
    CUtensorMap mXp, mPX, mFp, mPF, mRp, mLp;
    const unsigned long long* exp_tbl = nullptr;
    if (oz && !(ozmm_map(&mXp, ow.Xp, N, ow.ldX, N * ow.ldX, true) &&
                ozmm_map(&mPX, ow.PXp, b, ow.ldX, (int64_t)b * ow.ldX, false) &&
                ozmm_map(&mFp, ow.Fp, N, ow.ldF, N * ow.ldF, true) &&
                ozmm_map(&mPF, ow.PFp, b, ow.ldF, (int64_t)b * ow.ldF, false) &&
                ozmm_map(&mRp, ow.Rp, N, ow.ldR, N * ow.ldR, true) &&
                ozmm_map(&mLp, ow.Lp, b, ow.ldR, (int64_t)b * ow.ldR, false)))
        return KEVD_ECUDA;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double* Xd = static_cast<const double*>(X);
    double* Fd = static_cast<double*>(F);
    const float* Xf = static_cast<const float*>(X);
    float* Ff = static_cast<float*>(F);
    const int64_t ntiles = (N + kBM - 1) / kBM;
    const double inv_eps = 1.0 / eps;

    {
        TraceScope tr(kStOther, s);
        if (tc) {
            KEVD_CUDA_TRY(cudaMemsetAsync(pw.err, 0, sizeof(int), s));
            k_prepare<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(Xf, N, d, w, rho);
        } else {
            k_prepare<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(Xd, N, d, w, rho);
            if (oz) {
                KEVD_CUDA_TRY(kexp_table(s, &exp_tbl));
                k_xplanes<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(Xd, N, d, ow);
                KEVD_CUDA_TRY(cudaMemsetAsync(ow.flags, 0, sizeof(int), s));
            }
        }
    }
    KEVD_LAUNCH_CHECK();
    const size_t rej_smem = ((size_t)b * b + 3 * (size_t)b) * sizeof(double);   // H, L column, rho0, z
    KEVD_CUDA_TRY(cudaFuncSetAttribute(k_reject, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rej_smem));
    if (oz)
        KEVD_CUDA_TRY(cudaFuncSetAttribute(k_linv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)((size_t)b * b * sizeof(double))));
    const int rej_threads = b >= 32 ? 1024 : 128;
    const int tn = b <= 8 ? 1 : b <= 16 ? 2 : b <= 32 ? 4 : b <= 64 ? 8 : 16;
    switch (tn) {
        case 1: KEVD_CUDA_TRY(prepare_engine<1>()); break;
        case 2: KEVD_CUDA_TRY(prepare_engine<2>()); break;
        case 4: KEVD_CUDA_TRY(prepare_engine<4>()); break;
        case 8: KEVD_CUDA_TRY(prepare_engine<8>()); break;
        default: KEVD_CUDA_TRY(prepare_engine<16>()); break;
    }

    for (int rnd = 0; rnd < rounds; ++rnd) {
        {
            TraceScope tr(kStPropose, s);
            k_propose<<<1, 1024, 0, s>>>(w, rho, N, ntiles, b, r, greedy, opts->seed, rnd, proposals, opts->tol * N);
        }
        {
            TraceScope tr(kStGather, s);
            if (tc) k_gather<<<(unsigned)((d + r + 7) / 8), 256, 0, s>>>(w, Xf, (const float*)Ff, ldf, d, b);
            else k_gather<<<(unsigned)((d + r + 7) / 8), 256, 0, s>>>(w, Xd, (const double*)Fd, ldf, d, b);
        }
        {
            TraceScope tr(kStBlockH, s);
            k_blockH<<<(unsigned)((b * b + kBlockHWarps - 1) / kBlockHWarps), 32 * kBlockHWarps, 0, s>>>(w, d, b,
                                                                                                      inv_eps);
        }
        {
            TraceScope tr(kStReject, s);
            k_reject<<<1, rej_threads, rej_smem, s>>>(w, b, r, greedy, opts->seed, rnd, pivots);
        }
        if (tc) {
            TraceScope tr(kStEngine, s);
            KEVD_CUDA_TRY(launch_engine_tc(w, pw, Xf, Ff, ldf, rho, N, d, b, inv_eps, r, s));
        } else {
            if (oz) {
                {
                    // X X(S,:)^T and F(:, :k) F(S, :k)^T on the tensor cores at FP64 accuracy
                    TraceScope tp(kStProducts, s);
                    k_ozpanel<<<b, 128, 0, s>>>(w, ow, N, b);
                    KEVD_CUDA_TRY(launch_ozmm(mXp, mPX, ow.xe, 0, ow.pxe, 0, N, b, ow.ldX, w.st, w.Dx, w.ldD, 0,
                                              nullptr, 0, 0, ow.flags, s));
                    KEVD_CUDA_TRY(launch_ozmm(mFp, mPF, nullptr, 1, nullptr, 1, N, b, -3, w.st, w.Df, w.ldD, 0,
                                              nullptr, 0, 0, ow.flags, s));
                }
                TraceScope tr(kStEngine, s);
                // R = K(:, T) - F F(T,:)^T; G = R L^-T into F(:, k:k+m), on the tensor cores; rho
                k_rprep<<<(unsigned)((N + 31) / 32), 256, 0, s>>>(w, ow, N, inv_eps, exp_tbl);
                k_linv<<<1, 128, (size_t)b * b * sizeof(double), s>>>(w, ow, b);
                KEVD_CUDA_TRY(launch_ozmm(mRp, mLp, ow.re, 0, ow.le, 0, N, b, -2, w.st, Fd, ldf, ldf, ow.Fp, ow.ldF,
                                          N * ow.ldF, ow.flags, s));
                k_rho_update<<<(unsigned)((N + 63) / 64), 256, 0, s>>>(w, Fd, ldf, rho, N);
            } else {
                TraceScope tr(kStEngine, s);
                switch (tn) {
                    case 1: launch_engine<1>(w, Xd, Fd, ldf, rho, N, d, b, inv_eps, ntiles, s); break;
                    case 2: launch_engine<2>(w, Xd, Fd, ldf, rho, N, d, b, inv_eps, ntiles, s); break;
                    case 4: launch_engine<4>(w, Xd, Fd, ldf, rho, N, d, b, inv_eps, ntiles, s); break;
                    case 8: launch_engine<8>(w, Xd, Fd, ldf, rho, N, d, b, inv_eps, ntiles, s); break;
                    default: launch_engine<16>(w, Xd, Fd, ldf, rho, N, d, b, inv_eps, ntiles, s); break;
                }
            }
        }
        KEVD_LAUNCH_CHECK();
        if (opts->until_rank && (rnd % 8) == 7) {
            FactorState hs;
            KEVD_CUDA_TRY(cudaMemcpyAsync(&hs, w.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
            KEVD_CUDA_TRY(cudaStreamSynchronize(s));
            if (hs.done || hs.k + hs.m >= r) break;
        }
    }
    {
        TraceScope tr(kStOther, s);
        k_finalize<<<1, 1024, 0, s>>>(w, rho, N);
        const dim3 zg((unsigned)std::min<int64_t>((N + 255) / 256, 64), r);
        if (tc) k_zero_tail<<<zg, 256, 0, s>>>(w.st, Ff, ldf, N, r);
        else k_zero_tail<<<zg, 256, 0, s>>>(w.st, Fd, ldf, N, r);
    }
    KEVD_LAUNCH_CHECK();
    FactorState hs;
    int herr = 0;
    KEVD_CUDA_TRY(cudaMemcpyAsync(&hs, w.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    if (tc) KEVD_CUDA_TRY(cudaMemcpyAsync(&herr, pw.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (oz) KEVD_CUDA_TRY(cudaMemcpyAsync(&herr, ow.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    if (herr) return KEVD_ETIMEOUT;
    info->rank = hs.k;
    info->rounds = hs.rounds;
    info->trace_err = hs.final_sum;
    info->sum_m_sq = hs.sum_m_sq;
    info->sum_k = hs.sum_k;
    info->engine_rounds = hs.eng_rounds;
    if (hs.bad) return KEVD_EINVAL;
    return KEVD_OK;
}

extern "C" int rpchol_factor(const void* X, int x_dtype, int64_t N, int32_t d, double eps, int32_t r,
                             const kevd_opts* opts, void* F, int f_dtype, int64_t ldf, int64_t* pivots,
                             double* rho, int64_t* proposals, kevd_factor_info* info, void* workspace,
                             size_t ws_bytes, void* stream) {
    return rpchol_factor_impl(X, x_dtype, N, d, eps, r, opts, F, f_dtype, ldf, pivots, rho, proposals, info, workspace,
                              ws_bytes, stream, true);
}

// ===========================================================================
// Batched form: many independent problems (uneven N, d, eps, r, b) advance
// through Algorithm 2 in lockstep.  Every launch covers all problems (one grid
// dimension is the problem); the kernel-column engine is one persistent launch
// that walks a work list of (problem, 64-row tile) items.  The round loop is
// captured once into a CUDA graph (kevd_batch_create) and replayed
// (kevd_batch_run).  FP64 path, ARPC.
// ===========================================================================
namespace kevd {

struct BatchProb {
    const double* X;
    double* F;
    int64_t ldf;
    double* rho;
    int64_t* pivots;
    int64_t N;
    int d, r, b, rounds;
    double inv_eps;
    uint64_t seed;
    int64_t ntiles;
    FactorWs w;
};

__global__ void k_prepare_b(const BatchProb* __restrict__ P) {
    const BatchProb& p = P[blockIdx.y];
    if ((int64_t)blockIdx.x * blockDim.x >= p.N && blockIdx.x != 0) return;
    prepare_body(p.X, p.N, p.d, p.w, p.rho, blockIdx.x);
}

__global__ void __launch_bounds__(1024) k_propose_b(const BatchProb* __restrict__ P, int rnd) {
    const BatchProb& p = P[blockIdx.x];
    if (rnd >= p.rounds) {   // this problem has run its t = r/b rounds
        if (threadIdx.x == 0) {
            FactorState* st = p.w.st;
            if (st->m > 0) {
                st->sum_k += st->k;
                st->eng_rounds += 1;
            }
            st->k += st->m;
            st->kp += (st->m + 15) & ~15;
            st->sum_m_sq += (long long)st->m * st->m;
            st->m = 0;
            st->done = 1;
        }
        return;
    }
    propose_body(p.w, p.rho, p.N, p.ntiles, p.b, p.r, 0, p.seed, rnd, nullptr);
}

__global__ void k_gather_b(const BatchProb* __restrict__ P) {
    const BatchProb& p = P[blockIdx.y];
    gather_body(p.w, p.X, (const double*)p.F, p.ldf, p.d, p.b, blockIdx.x);
}

__global__ void k_blockH_b(const BatchProb* __restrict__ P) {
    const BatchProb& p = P[blockIdx.z];
    blockH_body(p.w, p.d, p.b, p.inv_eps, blockIdx.x * kBlockHWarps + (threadIdx.x >> 5));   // pairs past b*b return
}

__global__ void __launch_bounds__(1024) k_reject_b(const BatchProb* __restrict__ P, int rnd) {
    extern __shared__ double smem_rb[];
    const BatchProb& p = P[blockIdx.x];
    reject_body(p.w, p.b, p.r, 0, p.seed, rnd, p.pivots, smem_rb);
}

// Persistent engine over the work list; tile_off[q] = first item of problem q.
template <int TN>
__global__ void __launch_bounds__(256) k_engine_b(const BatchProb* __restrict__ P, const int64_t* __restrict__ tile_off,
                                                  int nprob) {
    extern __shared__ double smem_eb[];
    const int64_t total = tile_off[nprob];
    for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
        int lo = 0, hi = nprob - 1;   // last q with tile_off[q] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_off[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const BatchProb& p = P[lo];
        engine_body<TN>(p.w, p.X, p.F, p.ldf, p.rho, p.N, p.d, p.b, p.inv_eps, item - tile_off[lo], smem_eb);
    }
}

__global__ void __launch_bounds__(1024) k_finalize_b(const BatchProb* __restrict__ P) {
    const BatchProb& p = P[blockIdx.x];
    finalize_body(p.w, p.rho, p.N);
}

__global__ void k_zero_tail_b(const BatchProb* __restrict__ P) {
    const BatchProb& p = P[blockIdx.y];
    const int k = p.w.st->k;
    const int64_t cols = p.r - k;
    const int64_t total = cols * p.N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        p.F[(int64_t)(k + e / p.N) * p.ldf + e % p.N] = 0.0;
}

}  // namespace kevd

struct kevd_batch {
    int nprob;
    int rounds;
    int dmax, rmax, bmax;
    int64_t nmax;
    kevd::BatchProb* dprobs;   // device, in the caller's workspace (all problems)
    // engine groups by column-tile class TN (1, 2, 4, 8, 16): problems of a
    // group share one persistent engine launch per round
    struct Group {
        int tn;
        int n;
        kevd::BatchProb* probs;   // device copy of the group's descriptors
        int64_t* tile_off;        // device
    };
    std::vector<Group> groups;
    std::vector<kevd::FactorState*> states;
    cudaGraphExec_t exec;
    bool graph;
};

namespace {

static int tn_class(int b) { return b <= 8 ? 1 : b <= 16 ? 2 : b <= 32 ? 4 : b <= 64 ? 8 : 16; }

// layout: all descriptors | per group (<= 5): descriptors + tile offsets | per-problem factor workspaces
static size_t batch_layout(const kevd_problem* probs, int nprob, size_t* per_off) {
    using namespace kevd;
    size_t off = align_up(sizeof(BatchProb) * nprob);
    off += 5 * (align_up(sizeof(BatchProb) * nprob) + align_up(sizeof(int64_t) * (nprob + 1)));
    for (int q = 0; q < nprob; ++q) {
        size_t bytes = 0;
        carve_factor(nullptr, probs[q].N, probs[q].d, probs[q].r, probs[q].b, &bytes);
        if (per_off) per_off[q] = off;
        off += align_up(bytes);
    }
    return off;
}

template <int TN>
static int engine_group(const kevd_batch::Group& g, cudaStream_t s) {
    using namespace kevd;
    int nsm = 0, per_sm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KEVD_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return KEVD_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_engine_b<TN>, 256, engine_smem<TN>()) != cudaSuccess)
        return KEVD_ECUDA;
    const unsigned egrid = (unsigned)std::max(1, nsm * std::max(1, per_sm));
    k_engine_b<TN><<<egrid, 256, engine_smem<TN>(), s>>>(g.probs, g.tile_off, g.n);
    return KEVD_OK;
}

static int batch_enqueue_any(kevd_batch* h, cudaStream_t s) {
    using namespace kevd;
    const int np = h->nprob;
    k_prepare_b<<<dim3((unsigned)((h->nmax + 255) / 256), np), 256, 0, s>>>(h->dprobs);
    const size_t rej_smem = ((size_t)h->bmax * h->bmax + 3 * (size_t)h->bmax) * sizeof(double);
    for (int rnd = 0; rnd < h->rounds; ++rnd) {
        k_propose_b<<<np, 1024, 0, s>>>(h->dprobs, rnd);
        k_gather_b<<<dim3((unsigned)((h->dmax + h->rmax + 7) / 8), np), 256, 0, s>>>(h->dprobs);
        k_blockH_b<<<dim3((h->bmax * h->bmax + kBlockHWarps - 1) / kBlockHWarps, 1, np), 32 * kBlockHWarps, 0, s>>>(
            h->dprobs);
        k_reject_b<<<np, h->bmax >= 32 ? 1024 : 128, rej_smem, s>>>(h->dprobs, rnd);
        for (const auto& g : h->groups) {
            int st;
            switch (g.tn) {
                case 1: st = engine_group<1>(g, s); break;
                case 2: st = engine_group<2>(g, s); break;
                case 4: st = engine_group<4>(g, s); break;
                case 8: st = engine_group<8>(g, s); break;
                default: st = engine_group<16>(g, s); break;
            }
            if (st != KEVD_OK) return st;
        }
    }
    k_finalize_b<<<np, 1024, 0, s>>>(h->dprobs);
    k_zero_tail_b<<<dim3(64, np), 256, 0, s>>>(h->dprobs);
    return cudaGetLastError() == cudaSuccess ? KEVD_OK : KEVD_ECUDA;
}

template <int TN>
static cudaError_t batch_attrs() {
    using namespace kevd;
    return cudaFuncSetAttribute(k_engine_b<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)engine_smem<TN>());
}

}  // namespace

extern "C" size_t kevd_batch_workspace_bytes(const kevd_problem* probs, int nprob) {
    if (!probs || nprob < 1) return 0;
    for (int q = 0; q < nprob; ++q)
        if (probs[q].N < 1 || probs[q].d < 1 || probs[q].r < 1 || probs[q].b < 1 || probs[q].b > 128) return 0;
    return batch_layout(probs, nprob, nullptr);
}

extern "C" int kevd_batch_create(const kevd_problem* probs, int nprob, int use_graph, void* workspace,
                                 size_t ws_bytes, void* stream, kevd_batch** out) {
    using namespace kevd;
    if (!probs || nprob < 1 || !out) return KEVD_EINVAL;
    *out = nullptr;
    int bmax = 1, dmax = 1, rmax = 1, rounds = 0;
    int64_t nmax = 1;
    for (int q = 0; q < nprob; ++q) {
        const kevd_problem& p = probs[q];
        if (!p.X || !p.F || !p.pivots || !p.rho) return KEVD_EINVAL;
        if (p.N < 1 || p.d < 1 || p.r < 1 || p.r > p.N || p.ldf < p.N || p.b < 1 || p.b > 128 || p.r / p.b < 1)
            return KEVD_EINVAL;
        if (!(p.eps > 0.0) || !isfinite(p.eps)) return KEVD_EINVAL;
        bmax = std::max(bmax, p.b);
        dmax = std::max(dmax, p.d);
        rmax = std::max(rmax, p.r);
        nmax = std::max(nmax, p.N);
        rounds = std::max(rounds, p.r / p.b);
    }
    std::vector<size_t> offs(nprob);
    const size_t need = batch_layout(probs, nprob, offs.data());
    if (!workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return KEVD_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(workspace);
    kevd_batch* h = new kevd_batch();
    h->nprob = nprob;
    h->rounds = rounds;
    h->bmax = bmax;
    h->dmax = dmax;
    h->rmax = rmax;
    h->nmax = nmax;
    h->dprobs = reinterpret_cast<BatchProb*>(base);
    h->graph = use_graph != 0;
    h->exec = nullptr;
    std::vector<BatchProb> hp(nprob);
    for (int q = 0; q < nprob; ++q) {
        const kevd_problem& p = probs[q];
        BatchProb& b = hp[q];
        b.X = p.X;
        b.F = p.F;
        b.ldf = p.ldf;
        b.rho = p.rho;
        b.pivots = p.pivots;
        b.N = p.N;
        b.d = p.d;
        b.r = p.r;
        b.b = p.b;
        b.rounds = p.r / p.b;
        b.inv_eps = 1.0 / p.eps;
        b.seed = p.seed;
        b.ntiles = (p.N + kBM - 1) / kBM;
        size_t bytes = 0;
        b.w = carve_factor(base + offs[q], p.N, p.d, p.r, p.b, &bytes);
        h->states.push_back(b.w.st);
    }
    const size_t rej_smem = ((size_t)bmax * bmax + 3 * (size_t)bmax) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_reject_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rej_smem);
    bool ok = e == cudaSuccess &&
              cudaMemcpyAsync(h->dprobs, hp.data(), sizeof(BatchProb) * nprob, cudaMemcpyHostToDevice, s) == cudaSuccess;
    // engine groups
    std::vector<std::vector<BatchProb>> gp(5);
    std::vector<std::vector<int64_t>> gt(5, std::vector<int64_t>(1, 0));
    const int classes[5] = {1, 2, 4, 8, 16};
    for (int q = 0; q < nprob; ++q) {
        const int c = tn_class(hp[q].b);
        const int gi = c == 1 ? 0 : c == 2 ? 1 : c == 4 ? 2 : c == 8 ? 3 : 4;
        gp[gi].push_back(hp[q]);
        gt[gi].push_back(gt[gi].back() + hp[q].ntiles);
    }
    size_t goff = align_up(sizeof(BatchProb) * nprob);
    for (int gi = 0; gi < 5 && ok; ++gi) {
        kevd_batch::Group g;
        g.tn = classes[gi];
        g.n = (int)gp[gi].size();
        g.probs = reinterpret_cast<BatchProb*>(base + goff);
        g.tile_off = reinterpret_cast<int64_t*>(base + goff + align_up(sizeof(BatchProb) * nprob));
        goff += align_up(sizeof(BatchProb) * nprob) + align_up(sizeof(int64_t) * (nprob + 1));
        if (g.n == 0) continue;
        switch (g.tn) {
            case 1: e = batch_attrs<1>(); break;
            case 2: e = batch_attrs<2>(); break;
            case 4: e = batch_attrs<4>(); break;
            case 8: e = batch_attrs<8>(); break;
            default: e = batch_attrs<16>(); break;
        }
        ok = e == cudaSuccess &&
             cudaMemcpyAsync(g.probs, gp[gi].data(), sizeof(BatchProb) * g.n, cudaMemcpyHostToDevice, s) ==
                 cudaSuccess &&
             cudaMemcpyAsync(g.tile_off, gt[gi].data(), sizeof(int64_t) * (g.n + 1), cudaMemcpyHostToDevice, s) ==
                 cudaSuccess;
        h->groups.push_back(g);
    }
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
        delete h;
        return KEVD_ECUDA;
    }
    if (h->graph) {
        cudaStream_t cs = nullptr;
        cudaGraph_t g = nullptr;
        int st = KEVD_ECUDA;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            st = batch_enqueue_any(h, cs);
            if (cudaStreamEndCapture(cs, &g) != cudaSuccess) st = KEVD_ECUDA;
        }
        if (st == KEVD_OK && cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess) st = KEVD_ECUDA;
        if (g) cudaGraphDestroy(g);
        if (cs) cudaStreamDestroy(cs);
        if (st != KEVD_OK) {
            delete h;
            return st;
        }
    }
    *out = h;
    return KEVD_OK;
}

extern "C" int kevd_batch_run(kevd_batch* h, void* stream, kevd_factor_info* infos) {
    using namespace kevd;
    if (!h) return KEVD_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->graph) {
        TraceScope tr(kStOther, s);   // the whole batched round loop
        KEVD_CUDA_TRY(cudaGraphLaunch(h->exec, s));
    } else {
        TraceScope tr(kStOther, s);
        const int st = batch_enqueue_any(h, s);
        if (st != KEVD_OK) return st;
    }
    std::vector<FactorState> hs(h->nprob);
    for (int q = 0; q < h->nprob; ++q)
        KEVD_CUDA_TRY(cudaMemcpyAsync(&hs[q], h->states[q], sizeof(FactorState), cudaMemcpyDeviceToHost, s));
    KEVD_CUDA_TRY(cudaStreamSynchronize(s));
    trace_flush();
    int status = KEVD_OK;
    for (int q = 0; q < h->nprob; ++q) {
        if (infos) {
            infos[q].rank = hs[q].k;
            infos[q].rounds = hs[q].rounds;
            infos[q].trace_err = hs[q].final_sum;
            infos[q].sum_m_sq = hs[q].sum_m_sq;
            infos[q].sum_k = hs[q].sum_k;
            infos[q].engine_rounds = hs[q].eng_rounds;
            infos[q].reserved = 0;
        }
        if (hs[q].bad) status = KEVD_EINVAL;
    }
    return status;
}

extern "C" void kevd_batch_destroy(kevd_batch* h) {
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    delete h;
}
