/*
 * kevd.h -- C-ABI of the GB300 (sm_103a) implementation of the low-rank
 * eigendecomposition of bistochastic kernel matrices of Vales & Giannakis,
 * "Accelerated decomposition of bistochastic kernel matrices by low rank
 * approximation" (arXiv 2510.26574).
 *
 * The three stages of Algorithm 1 are three calls:
 *
 *   rpchol_factor      partial Cholesky factor F (N x r) of the implicit
 *                      Gaussian kernel matrix K_ij = exp(-|x_i - x_j|^2 / eps),
 *                      by greedy pivoting or by accelerated randomly pivoted
 *                      Cholesky (Algorithm 2 with the check of Algorithm 3).
 *                      K is never formed: at most N(r+1) entries are evaluated.
 *   bistoch_normalize  degree vectors d~ = F F^T 1 and q~ = F F^T d~^-1
 *                      (Algorithm 1, with its positivity checks) and the two
 *                      weighted r x r Gram matrices A = F^T D~^-2 F and
 *                      C = F^T Q~^-1 F (Section 2.2: B = D~^-1 F, C).
 *   eig_topk           top-k eigenpairs of P~ = B C B^T (Section 2, the B C B^T
 *                      method): orthonormal basis of range(B) from the EVD of
 *                      A = B^T B, r x r EVD of the inner matrix, lift
 *                      U = D~^-1 F Y to N x k.
 *
 * rpchol_factor_lowmem, bistoch_normalize_lowmem and eig_topk_lowmem are the
 * same three stages with F kept as its pivots and r x r block W = F(S,:)
 * (the low-memory variant of Appendix A), rebuilding rows of F from X.
 *
 * Conventions shared by every call:
 *  - All array arguments are DEVICE pointers unless marked "host".  The
 *    caller allocates and owns every buffer, including the workspace; the
 *    library allocates no device memory on these paths and frees nothing.
 *  - Matrices are column-major with an explicit leading dimension
 *    (F: N x r, ldf >= N; A, C: rank x rank, ld = rank; U: N x k, ld = N).
 *    X is row-major N x d (point i occupies X[i*d .. i*d+d-1]).
 *  - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default).
 *    Each call synchronises that stream once before returning, to read its
 *    host outputs and error flags; device outputs are complete on return.
 *  - Return value: a KEVD_* status.  On a non-zero status the device outputs
 *    are unspecified.  Argument errors are detected before any work is
 *    enqueued.
 *  - workspace must be at least kevd_workspace_bytes(...) bytes, 256-byte
 *    aligned, and must not be used concurrently by another call.
 */
#ifndef KEVD_H
#define KEVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define KEVD_OK 0
#define KEVD_EINVAL 1      /* invalid argument, or non-finite value in X        */
#define KEVD_ED_NONPOS 2   /* some d~_i <= 0 (Algorithm 1, first assert)         */
#define KEVD_EQ_NONPOS 3   /* some q~_i <= 0 (Algorithm 1, second assert)        */
#define KEVD_ECUDA 4       /* a CUDA runtime or cuSOLVER call failed             */
#define KEVD_EWORKSPACE 5  /* workspace missing, misaligned or too small         */
#define KEVD_ETIMEOUT 6    /* a bounded device-side wait gave up (about 1 s)     */
#define KEVD_EEIG 7        /* the r x r symmetric eigensolver did not converge   */
#define KEVD_ESCRATCH 8    /* problem needs more than the static scratch of      */
                           /* rpchol_factor_noalloc                              */

/* element types */
#define KEVD_F64 0
#define KEVD_F32 1

/* pivot rules (Appendix A) */
#define KEVD_GREEDY 0      /* s = argmax rho, one pivot per round (b = 1)      */
#define KEVD_ARPC 1        /* Algorithm 2 + Algorithm 3, blocks of b proposals */

/* arithmetic of the kernel-column engine (Algorithm 2, line computing G) */
#define KEVD_PREC_FP64 0   /* X, F, all products in FP64                       */
#define KEVD_PREC_BF16X3 1 /* X, F in FP32; products on the tensor cores as     */
                           /* hi*hi + hi*lo + lo*hi of BF16 halves, FP32 sums;  */
                           /* rho, H, reject and L in FP64                      */

/* which call kevd_workspace_bytes sizes */
#define KEVD_WS_FACTOR 0
#define KEVD_WS_NORMALIZE 1
#define KEVD_WS_EIG 2
#define KEVD_WS_FIX 3      /* constant_eigvec_fix: N and k                      */
#define KEVD_WS_LOWMEM_FACTOR 4     /* rpchol_factor_lowmem: N, d, r, opts     */
#define KEVD_WS_LOWMEM_NORMALIZE 5  /* bistoch_normalize_lowmem: N, d, rank    */
#define KEVD_WS_LOWMEM_EIG 6        /* eig_topk_lowmem: N, d, rank, k          */

typedef struct kevd_opts {
    int32_t mode;        /* KEVD_GREEDY or KEVD_ARPC                                   */
    int32_t precision;   /* KEVD_PREC_*                                                */
    int32_t block_b;     /* ARPC block size b, 1..128 (greedy uses b = 1)              */
    int32_t until_rank;  /* 0: t = floor(r/b) rounds, as in Algorithm 2;               */
                         /* 1: rounds continue until exactly r pivots are accepted     */
    int32_t max_rounds;  /* cap on rounds when until_rank = 1 (0: 4*ceil(r/b) + 16)    */
    int32_t reserved;    /* must be 0                                                  */
    uint64_t seed;       /* Philox4x32-10 key for proposals (stream 0) and z (stream 1)*/
    double tol;          /* ARPC stops once sum(rho) <= tol * N, 0 <= tol < 1 (0: only */
                         /* at sum(rho) = 0, Appendix A).  A floor at the arithmetic's  */
                         /* resolution (~1e-6 for FP32 factors) keeps noise-level       */
                         /* pivots out of F when r exceeds the numerical rank of K      */
} kevd_opts;

/*
 * kevd_opts_init -- the documented defaults for `precision` (KEVD_PREC_*):
 * ARPC, b = 64, t = floor(r/b) rounds, seed 0, and the stopping floor tol =
 * 1e-6 for KEVD_PREC_BF16X3 (0, the paper's rule, for KEVD_PREC_FP64).  A
 * zero-initialised kevd_opts has tol = 0, which lets an FP32 factor run past
 * the kernel's numerical rank on noise-level pivots (d~ may then come out
 * non-positive); start from this call and change the fields you need.
 * Not part of the paper.  Never fails; a NULL o is ignored.
 */
void kevd_opts_init(kevd_opts* o, int32_t precision);

typedef struct kevd_factor_info {
    int32_t rank;        /* accepted pivots = columns of F written (<= r)               */
    int32_t rounds;      /* rounds executed                                             */
    double trace_err;    /* sum(rho) = tr(K - F F^T) after the last round (Appendix A)  */
    int64_t sum_m_sq;    /* sum over rounds of (pivots accepted in the round)^2.  The   */
                         /* engine's arithmetic is N (2 d rank + rank^2) flops, of      */
                         /* which N (rank^2 - sum_m_sq) are the products with the F     */
                         /* columns of earlier rounds and N sum_m_sq the solves with L  */
    int64_t sum_k;       /* sum over engine rounds of the rank before the round; the    */
                         /* engine reads e N (sum_k + d engine_rounds) bytes of F and X */
    int32_t engine_rounds; /* rounds that accepted at least one pivot                   */
    int32_t reserved;
} kevd_factor_info;

/* tracing stages (kevd_trace_read index) */
#define KEVD_STAGE_PROPOSE 0   /* pivot proposal / argmax                    */
#define KEVD_STAGE_GATHER 1    /* gather of proposal rows                    */
#define KEVD_STAGE_BLOCKH 2    /* H = K(S',S') - F_S' F_S'^T                 */
#define KEVD_STAGE_REJECT 3    /* Algorithm 3                                */
#define KEVD_STAGE_ENGINE 4    /* kernel-column engine + residual update     */
#define KEVD_STAGE_DEGREE 5    /* d~, q~                                     */
#define KEVD_STAGE_GRAM 6      /* weighted Gram matrices A, C                */
#define KEVD_STAGE_SOLVER 7    /* r x r symmetric eigensolves                */
#define KEVD_STAGE_LIFT 8      /* U = D~^-1 F Y                              */
#define KEVD_STAGE_OTHER 9     /* set-up, reductions, small products         */
#define KEVD_STAGE_PRODUCTS 10 /* FP64 path: the engine's X X(S,:)^T and      */
                               /* F F(S,:)^T on the tensor cores (the engine  */
                               /* stage then holds exp, L solve and rho)      */
#define KEVD_NUM_STAGES 11

/*
 * rpchol_factor -- pivoted partial Cholesky of the implicit Gaussian kernel
 * matrix (Section 1.2; Appendix A, Algorithms 2 and 3; kernel of Eq.
 * (data-kernel) with the delay factor J folded into eps).
 * With KEVD_PREC_FP64 the engine's products X X(S,:)^T and F F(S,:)^T run on
 * the tensor cores at FP64 accuracy (six-digit BF16 slices summed exactly),
 * when X's rows have an even length, ldf is even and X, F are 16-byte
 * aligned; otherwise, or with KEVD_ENGINE=fp64 in the environment, on the FP64
 * pipe.  Both agree to rounding (1e-10 in F); kevd_workspace_bytes must be
 * queried under the same environment.
 *
 *   X         device, N x d row-major, element type x_dtype (KEVD_F64 for
 *             KEVD_PREC_FP64, KEVD_F32 for KEVD_PREC_BF16X3).
 *   eps       bandwidth, finite and > 0.
 *   r         maximum rank, 1 <= r <= N.
 *   opts      host; mode, b, seed, rounds rule.  Greedy ignores b (uses 1).
 *   F         device, N x r column-major (ldf >= N), element type f_dtype
 *             (the type of X).  Columns [0, rank) receive the factor, in acceptance
 *             order; columns [rank, r) are set to zero.
 *   pivots    device int64[r]; entries [0, rank) receive the accepted pivots
 *             in acceptance order, so F(pivots, :) is lower triangular.
 *   rho       device double[N]; receives the residual diagonal diag(K - F F^T),
 *             clamped at 0.
 *   proposals optional device int64[rounds_max * b] (NULL to skip): the
 *             proposals of round i at [i*b, i*b + b), in draw order (ARPC), or
 *             the argmax pivot (greedy, b = 1).  rounds_max = floor(r/b) (r for
 *             greedy), or the max_rounds rule when until_rank = 1.
 *   info      host; receives rank, rounds and sum(rho).
 *
 * Sampling (the paper leaves the random source open): proposal j of round i is
 * the smallest index n with cumsum(rho)_n > u * sum(rho), u the 53-bit uniform
 * of Philox4x32-10 with key = seed and counter (j, i, 0, 0); the accept test of
 * Algorithm 3 for position j uses counter (j, i, 1, 0).  A proposal is accepted
 * iff H(j,j) > 0 and z * rho0(j) < H(j,j).  Rounds stop early once sum(rho) = 0
 * (or falls to opts->tol * N).
 * Errors: KEVD_EINVAL (bad argument, or a non-finite coordinate in X, reported
 * after the factorisation ran), KEVD_EWORKSPACE, KEVD_ECUDA, KEVD_ETIMEOUT
 * (precision form: a tensor-core pipeline wait gave up; outputs unspecified).
 */
int rpchol_factor(const void* X, int x_dtype, int64_t N, int32_t d, double eps, int32_t r,
                  const kevd_opts* opts, void* F, int f_dtype, int64_t ldf,
                  int64_t* pivots, double* rho, int64_t* proposals, kevd_factor_info* info,
                  void* workspace, size_t ws_bytes, void* stream);

/*
 * rpchol_factor_noalloc -- rpchol_factor without a workspace argument.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc, e.g. a plugin whose host application owns all device memory
 * through its own pool, or a process that may not allocate device memory after
 * start-up.  It allocates nothing and calls no allocating routine.
 *
 * The workspace is a file-scope device array of KEVD_NOALLOC_SCRATCH_BYTES
 * (16 MiB) that every GPU which loads the library holds until the process
 * exits.  Sizes whose kevd_workspace_bytes(KEVD_WS_FACTOR, N, d, r, 1, opts)
 * exceeds it are rejected with KEVD_ESCRATCH before any device work (about
 * N <= 1.8 million at d = 64, r = 1,024, b = 64).  Every call looks up the
 * array's device address (cudaGetSymbolAddress, which allocates nothing) on
 * the caller's current device.  All calls share the one array and each starts
 * by re-initialising what it reads, so back-to-back calls are fine, but calls
 * that overlap on the GPU (other streams, other host threads) race on it.
 * Like rpchol_factor it reads its results back and synchronises `stream`, so
 * it cannot be recorded into a CUDA graph by stream capture.  With tracing on
 * (kevd_trace_enable) the tracer creates CUDA events; that is the only
 * resource it may create.  Arguments, outputs and statuses are those of
 * rpchol_factor; both precision forms are accepted.  The FP64 form keeps the
 * engine's products on the FP64 pipe (the tensor-core form's two N x b product
 * arrays would not fit the array), so its outputs equal rpchol_factor's under
 * KEVD_ENGINE=fp64.
 */
#define KEVD_NOALLOC_SCRATCH_BYTES (16u << 20)
int rpchol_factor_noalloc(const void* X, int x_dtype, int64_t N, int32_t d, double eps, int32_t r,
                          const kevd_opts* opts, void* F, int f_dtype, int64_t ldf,
                          int64_t* pivots, double* rho, int64_t* proposals, kevd_factor_info* info,
                          void* stream);

/*
 * bistoch_normalize -- degree vectors and weighted Gram matrices of the
 * bistochastic normalisation (Section 2.2; Algorithm 1, lines forming D~ and
 * Q~ with their asserts; Section 2: B = D~^-1 F, C = F^T Q~^-1 F).
 *
 *   F      device, N x rank column-major (ldf >= N), element type f_dtype.
 *   dtil   device double[N]: d~ = F (F^T 1).
 *   qtil   device double[N]: q~ = F (F^T d~^-1).
 *   A      device double[rank*rank], column-major: F^T diag(d~)^-2 F.
 *   C      device double[rank*rank], column-major: F^T diag(q~)^-1 F.
 * Both Gram matrices are exactly symmetric (one triangle is computed and
 * mirrored).  FP64 F: FP64 products.  FP32 F: degree vectors from FP32
 * products summed in FP64 per block of columns; Grams from FP32 products with
 * FP32 sums per row split (round to nearest), reduced across splits in FP64.
 * Errors: KEVD_ED_NONPOS if some d~_i <= 0 (A, C, q~ unspecified),
 * KEVD_EQ_NONPOS if some q~_i <= 0, KEVD_EINVAL, KEVD_EWORKSPACE, KEVD_ECUDA,
 * KEVD_ETIMEOUT.
 */
int bistoch_normalize(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf,
                      double* dtil, double* qtil, double* A, double* C,
                      void* workspace, size_t ws_bytes, void* stream);

/*
 * eig_topk -- top-k eigenpairs of P~ = B C B^T, B = D~^-1 F (Section 2 and
 * Section 2.2; Algorithm 1 lines computing the QR, the r x r EVD and U = Q1 V).
 * Two routes to the orthonormal basis of range(B):
 *   Cholesky (taken when A = B^T B is numerically positive definite):
 *     A = R^T R (cuSOLVER potrf), Q1 = B R^-1, inner matrix M = R C R^T
 *     (formed FP64-accurate on the tensor cores from digit planes), M =
 *     V Lambda V^T, U = D~^-1 F Y with Y = R^-1 V_k.  The top-k of M comes
 *     from the subset eigensolver (cuSOLVER syevdx) for FP64 F.  For FP32 F
 *     with b = 2k + 32 <= rank / 3, it comes from block subspace iteration:
 *     b columns, six power steps, Rayleigh-Ritz, more steps when the
 *     observed rate allows.  That path accepts only when every returned pair
 *     has |M v - theta v| <= 1e-6 theta (each eigenvalue within 1e-6
 *     relative), and otherwise falls back to syevdx.  kept = rank.
 *   spectral (when potrf reports A singular): the EVD A = W S W^T, Q1 =
 *     B W S^-1/2 on the directions kept; directions with S_j <= tau * max(S)
 *     are dropped (this replaces the paper's regularisation of the QR by
 *     gamma, Section 4.1).  Then M = S^1/2 W^T C W S^1/2 = V Lambda V^T and
 *     Y = W S^-1/2 V.
 *
 *   F, dtil, A, C  as produced by the two calls above (rank x rank Grams).
 *   k              number of eigenpairs, 1 <= k <= rank.
 *   tau            relative cutoff of the spectral route, 0 <= tau < 1 (1e-13
 *                  suits FP64).
 *   evals          device double[k]: eigenvalues, descending.
 *   U              device double[N*k], column-major, ld = N: orthonormal
 *                  eigenvectors; each column is signed so that its entry of
 *                  largest magnitude (lowest index on ties) is positive.
 *   kept           optional host int32*: number of Gram directions kept.
 * Environment (comparisons and tests): KEVD_TOPK=full takes the subset
 * eigensolver on both forms; KEVD_TOPK=subspace requires the subspace path
 * (KEVD_EEIG when it does not apply or its check fails, instead of the
 * fallback); KEVD_SYEV=native takes this library's own top-k eigensolver.
 * Errors: KEVD_EINVAL, KEVD_EWORKSPACE, KEVD_EEIG, KEVD_ETIMEOUT (a bounded
 * wait of a tensor-core product gave up), KEVD_ECUDA.
 */
int eig_topk(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf,
             const double* dtil, const double* A, const double* C, int32_t k, double tau,
             double* evals, double* U, int32_t* kept,
             void* workspace, size_t ws_bytes, void* stream);

/*
 * symmetric_normalize, symmetric_eig_topk -- the symmetric normalisation
 * L~ = D~^-1/2 F F^T D~^-1/2 (Section 2.1), whose inner matrix is C = I: the
 * top-k eigenpairs are those of A_s = (D~^-1/2 F)^T (D~^-1/2 F) = F^T D~^-1 F
 * (the SVD form the section describes), lifted by U = D~^-1/2 F V Lambda^-1/2.
 *   symmetric_normalize: dtil (device double[N]) = F F^T 1 (KEVD_ED_NONPOS if
 *   some entry <= 0), As (device double[rank*rank], column-major, exactly
 *   symmetric).  Workspace: kevd_workspace_bytes(KEVD_WS_NORMALIZE, ...).
 *   symmetric_eig_topk: evals (device double[k], descending) and U (device
 *   double[N*k], column-major, sign convention as eig_topk).  Workspace:
 *   kevd_workspace_bytes(KEVD_WS_EIG, ...).  Errors: KEVD_EINVAL,
 *   KEVD_EWORKSPACE, KEVD_EEIG, KEVD_ETIMEOUT (the lift's tensor-core product
 *   gave up a bounded wait), KEVD_ECUDA.
 */
int symmetric_normalize(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf, double* dtil,
                        double* As, void* workspace, size_t ws_bytes, void* stream);
int symmetric_eig_topk(const void* F, int f_dtype, int64_t N, int32_t rank, int64_t ldf,
                       const double* dtil, const double* As, int32_t k, double* evals, double* U,
                       void* workspace, size_t ws_bytes, void* stream);

/*
 * constant_eigvec_fix -- the optional last lines of Algorithm 1: set the first
 * column of U (device, N x k column-major, ld = N) to 1_N / sqrt(N) and
 * re-orthonormalise the columns in place (CholeskyQR applied twice: the
 * result equals the Q of a QR factorisation with positive diagonal R).
 * Workspace: kevd_workspace_bytes(KEVD_WS_FIX, N, 0, k, k, NULL).  Errors:
 * KEVD_EINVAL, KEVD_EWORKSPACE, KEVD_EEIG (columns numerically dependent),
 * KEVD_ECUDA.
 */
int constant_eigvec_fix(double* U, int64_t N, int32_t k, void* workspace, size_t ws_bytes, void* stream);

/*
 * Low-memory form (Appendix A, closing paragraph; Remark of Section 4.2: ARPC
 * keeping only an r x r factor of F and recomputing its other entries when
 * needed).  FP64 only.  The factor is the pivot list S and W = F(S,:), the
 * rank x rank lower triangular Cholesky factor of K(S,S); every row of F is
 * F(i,:) = K(i,S) W^-T.  No N x r array is stored: the N-long passes form the
 * kernel values K(panel, S) of a row panel of P rows at a time, with
 * P = min(N rounded up to 64, max(64, floor(2^24 / r) rounded down to 64))
 * (at most 128 MiB of panel; KEVD_LOWMEM_PANEL=rows in the environment
 * lowers floor(2^24 / r) but cannot raise it, and kevd_workspace_bytes must be
 * queried under the same setting), so the workspace is O(N + r d + P r + r b)
 * doubles.  Each round of the factor, each of the three normalisation passes
 * and the lift recompute the kernel values they need: about
 * N d (r^2 / (2 b) + 4 r) multiply-adds beyond the stored-F path, plus one
 * triangular solve of N rows against W (N r^2 / 2) in the normalisation.
 *
 * rpchol_factor_lowmem -- Algorithms 2 and 3 as rpchol_factor (same sampling,
 * Philox streams, acceptance rule, stopping rules and per-round decisions up
 * to rounding), with F replaced by (S, W).
 *   X, N, d, eps, r, opts, pivots, rho, proposals, info  as rpchol_factor
 *             (X is FP64 and opts->precision must be KEVD_PREC_FP64).
 *   W         device, r x r column-major, ldw >= r: rows and columns
 *             [0, rank) receive F(pivots, :) (lower triangular); the rest of
 *             the r x r block is set to zero.
 *   The host synchronises with `stream` once per round to read the rank.
 *   Errors as rpchol_factor.
 *
 * bistoch_normalize_lowmem -- the outputs of bistoch_normalize for the factor
 * F = K(:,S) W^-T, from (X, S, W) in three passes over the panels:
 * d~ = K(:,S) y with y = W^-T W^-1 K(S,:) 1, q~ = K(:,S) z with
 * z = W^-T W^-1 K(S,:) d~^-1, and the Grams from the rebuilt panels
 * F_p = K(p,S) W^-T (a triangular solve per panel).
 *   pivots    device int64[rank]; an index outside [0, N) gives KEVD_EINVAL.
 *   W, ldw    the factor's W (its leading rank x rank block).
 *   dtil, qtil, A, C, errors  as bistoch_normalize.
 *
 * eig_topk_lowmem -- eig_topk for the same factor: the r x r stage is
 * eig_topk's; the lift is U = D~^-1 K(:,S) (W^-T Y) per panel.  N <= 2^31 - 1.
 *   Arguments as eig_topk, with (X, N, d, eps, pivots, W, ldw) in place of F.
 */
int rpchol_factor_lowmem(const double* X, int64_t N, int32_t d, double eps, int32_t r,
                         const kevd_opts* opts, double* W, int64_t ldw, int64_t* pivots,
                         double* rho, int64_t* proposals, kevd_factor_info* info,
                         void* workspace, size_t ws_bytes, void* stream);
int bistoch_normalize_lowmem(const double* X, int64_t N, int32_t d, double eps, const int64_t* pivots,
                             const double* W, int64_t ldw, int32_t rank, double* dtil, double* qtil,
                             double* A, double* C, void* workspace, size_t ws_bytes, void* stream);
int eig_topk_lowmem(const double* X, int64_t N, int32_t d, double eps, const int64_t* pivots,
                    const double* W, int64_t ldw, int32_t rank, const double* dtil, const double* A,
                    const double* C, int32_t k, double tau, double* evals, double* U, int32_t* kept,
                    void* workspace, size_t ws_bytes, void* stream);

/*
 * kevd_kernel_exp -- the exponential the FP64 engine on the tensor cores uses
 * for the Gaussian kernel values exp(-|x_i - x_s|^2 / eps) of Algorithm 2: out[i]
 * = exp(t[i]) for t[i] <= 0 within one ulp, 0 for t[i] <= -708 (a
 * table-driven method with its polynomial in fixed point, so that it runs on
 * the integer pipe).  t, out: device double[n] (out may alias t).  Enqueued on
 * `stream`; the first call on a device uploads an 8 KiB table and waits for it.
 * Returns KEVD_EINVAL for NULL pointers or n < 0.
 */
int kevd_kernel_exp(const double* t, int64_t n, double* out, void* stream);

/*
 * kevd_workspace_bytes -- bytes of workspace the call `which`
 * (KEVD_WS_*) needs for these sizes (d only matters for the factors and the
 * low-memory calls, k only for the eigen calls; opts may be NULL except for
 * the two factors).  KEVD_WS_NORMALIZE sizes for an FP64 factor, whose
 * tensor-core Grams keep the digit planes of one slab of rows (at most 6 GiB),
 * unless opts->precision is KEVD_PREC_BF16X3 (an FP32 factor: no planes).
 * Returns 0 for invalid sizes.  The KEVD_WS_EIG and
 * KEVD_WS_LOWMEM_EIG sizes query the eigensolver and therefore need a CUDA
 * device.
 */
size_t kevd_workspace_bytes(int which, int64_t N, int32_t d, int32_t r, int32_t k,
                            const kevd_opts* opts);

/*
 * Batched form (no counterpart in the paper; its method applied to many
 * independent problems at once).  Problems of uneven N, d, eps, r and b run
 * Algorithm 2 (ARPC, FP64) in lockstep: every launch covers all problems and
 * the kernel-column engine is one persistent launch over a work list of
 * (problem, 64-row tile) items.  kevd_batch_create uploads the problem table
 * into the caller's workspace and, with use_graph = 1, captures the whole
 * round loop into a CUDA graph once; kevd_batch_run replays it (or enqueues
 * the launches) on `stream`, waits, and fills one kevd_factor_info per
 * problem.  Each problem's outputs equal, bit for bit, those of rpchol_factor
 * with the same arguments (mode ARPC, precision FP64, t = floor(r/b) rounds)
 * and the engine's products on the FP64 pipe (KEVD_ENGINE=fp64).  The handle
 * owns no device memory; the workspace and every problem buffer must outlive
 * it, and the problem table is read only at creation.
 */
typedef struct kevd_problem {
    const double* X;     /* device, N x d row-major                        */
    int64_t N;
    int32_t d;
    int32_t r;           /* 1 <= r <= N                                    */
    int32_t b;           /* 1..128, floor(r/b) >= 1                         */
    int32_t reserved;
    double eps;
    uint64_t seed;
    double* F;           /* device, N x r column-major, ld = ldf >= N       */
    int64_t ldf;
    int64_t* pivots;     /* device int64[r]                                  */
    double* rho;         /* device double[N]                                 */
} kevd_problem;

typedef struct kevd_batch kevd_batch;

size_t kevd_batch_workspace_bytes(const kevd_problem* probs, int nprob);
int kevd_batch_create(const kevd_problem* probs, int nprob, int use_graph, void* workspace, size_t ws_bytes,
                      void* stream, kevd_batch** out);
int kevd_batch_run(kevd_batch* batch, void* stream, kevd_factor_info* infos);
void kevd_batch_destroy(kevd_batch* batch);

/*
 * Tracing (not part of the paper; the stage timing the measurements use).
 * kevd_trace_enable(1) makes every later call record a CUDA event pair on its
 * stream around each stage's launches; the elapsed times are folded into
 * per-stage totals when the call synchronises.  kevd_trace_read copies the
 * accumulated milliseconds and launch-group counts of the first n stages into
 * host arrays; kevd_trace_reset zeroes them.  kevd_trace_enable returns the
 * previous setting.  Tracing adds event records only; results are unchanged.
 */
int kevd_trace_enable(int on);
void kevd_trace_reset(void);
int kevd_trace_read(double* ms, int64_t* launches, int n);

/* kevd_status_string -- static, human-readable text of a status code. */
const char* kevd_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* KEVD_H */
