// Device state and workspace layout of rpchol_factor, shared by its FP64
// kernels (factor.cu) and the tensor-core engine of the precision form
// (engine_tc.cu).
#pragma once
#include "common.cuh"

namespace kevd {

constexpr int kBM = 64;   // rows per engine tile = rho tile of the sampler
constexpr int kBK = 16;   // inner-dimension chunk of the engine

struct FactorState {
    int32_t k;        // committed rank
    int32_t m;        // accepted in the current round
    int32_t rounds;   // rounds executed
    int32_t done;     // 1 once sum(rho) = 0, the rank cap is reached, or greedy stops
    int32_t bad;      // non-finite coordinate seen in X
    int32_t kp;       // padded rank: sum over rounds of m rounded up to 16 (the tensor-core
                      // FP64 engine's column offset of each round in the digit planes of F)
    double total;     // sum(rho) seen by the last proposal step
    double final_sum; // sum(rho) after the last round
    long long sum_m_sq; // sum over rounds of m^2
    long long sum_k;    // sum over rounds with m > 0 of the rank before the round
    int32_t eng_rounds; // rounds with m > 0
    int32_t pad2;
};

struct FactorWs {
    FactorState* st;
    double* xn;        // N: |x_i|^2
    double* tile_sum;  // ntiles: sum of rho over the tile
    double* tile_max;  // ntiles: max rho over the tile
    int64_t* tile_idx; // ntiles: lowest index attaining tile_max
    double* pre_incl;  // ntiles: inclusive prefix of tile_sum
    double* pre_excl;  // ntiles: exclusive prefix of tile_sum
    int64_t* prop;     // b: proposals of the round
    int32_t* acc_pos;  // b: accepted positions into prop
    int32_t* tpos;     // b: scratch of k_reject
    double* XSP;       // d x b: X(prop, :)^T
    double* FSP;       // r x b: F(prop, :)^T
    double* xnS;       // b: |x_prop|^2
    double* H;         // b x b
    double* Lfull;     // b x b: L columns at proposal positions
    double* Lc;        // b x b: compact L(T, T), row-major, ld = b
    // FP64 path with the products on the tensor cores (null otherwise):
    double* Dx;        // ldD x b: X X(S,:)^T of the round, column l = accepted pivot l
    double* Df;        // ldD x b: F(:, :k) F(S, :k)^T
    int64_t ldD;
    double* fm;        // N: running max over the columns written so far of |F(i, :)|
};

// Panels of the tensor-core products of the FP64 path (host-launched kernels only).
// Workspace of the FP64 engine on the tensor cores (ozmm.cu): seven-digit BF16
// planes (plane s of an R x ldk operand at s R ldk, row i at i ldk, K-major)
// and their row exponents.
struct OzWs {
    uint16_t* Xp;      // X: N x ldX, exponents xe (once per factorisation)
    int* xe;
    uint16_t* Fp;      // F: N x ldF, exponent 1 for every row; round t's columns at
                       // [kp_t, kp_t + m_t), zero up to kp_t + round16(m_t)
    uint16_t* Rp;      // R = K(:, T) - F F(T, :)^T: N x ldR, exponents re
    int* re;
    uint16_t* PXp;     // X(S, :): b x ldX, exponents pxe (rows past m zero)
    int* pxe;
    uint16_t* PFp;     // F(S, :): b x ldF (rows past m zero)
    uint16_t* Lp;      // L(T,T)^-1: b x ldR, exponents le (rows and columns past m zero)
    int* le;
    double* Linv;      // b x ldLi FP64 scratch of the inverse
    int* flags;        // bit 2: a bounded wait gave up
    int ldX, ldF, ldR, ldLi;
};



// Extra workspace of the precision form (BF16 hi/lo split operands).
struct PanelWs {
    uint16_t* panel;   // nchunk_max x 2 (hi, lo) x BN x 64 bf16, K-major, 128-byte swizzled
    float* Lf;         // BN x BN: L(T,T) in FP32, row-major, zero past m
    float* nS;         // BN: |x_s|^2 of the accepted pivots (FP32)
    int64_t* pidx;     // BN: row index of accepted pivot l (-1 past m)
    int* err;          // device-side wait timeout flag
};

constexpr int kTcBM = 128;   // rows per tensor-core tile (UMMA M)
constexpr int kTcBK = 64;    // K elements per staged chunk (one 128-byte swizzle row of bf16)

inline int tc_chunks(int d, int r) { return (d + kTcBK - 1) / kTcBK + (r + kTcBK - 1) / kTcBK; }

// Round launchers of the FP64 path (factor.cu), also used by the low-memory
// factor (lowmem.cu): workspace layout, a1 set-up, a2 proposals, a3 H, a4
// Algorithm 3, and the final commit with sum(rho).
FactorWs carve_factor_fp64(void* base, int64_t N, int d, int r, int b, size_t* bytes);
void launch_prepare_fp64(const double* X, int64_t N, int d, const FactorWs& w, double* rho, cudaStream_t s);
void launch_propose(const FactorWs& w, const double* rho, int64_t N, int b, int r, int greedy, uint64_t seed, int rnd,
                    int64_t* proposals, double floor_sum, cudaStream_t s);
void launch_blockH(const FactorWs& w, int d, int b, double inv_eps, cudaStream_t s);
cudaError_t launch_reject(const FactorWs& w, int b, int r, int greedy, uint64_t seed, int rnd, int64_t* pivots,
                          cudaStream_t s);
void launch_finalize(const FactorWs& w, const double* rho, int64_t N, cudaStream_t s);

// Host launcher of the tensor-core engine (engine_tc.cu).
cudaError_t launch_engine_tc(const FactorWs& w, const PanelWs& p, const float* X, float* F, int64_t ldf,
                             double* rho, int64_t N, int d, int b, double inv_eps, int r, cudaStream_t s);

}  // namespace kevd
