// FP64-accurate tensor-core products C = A B^T along rows (ozgemm.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "factor.cuh"

namespace kevd {

// True when a 16-byte aligned FP64 matrix with leading dimension ld (even) can
// be described by a TMA tensor map.
bool ozgemm_layout_ok(const double* p, int64_t ld);

// C(i, j) = sum_{c < K} A(i, c) B(j, c) (divided by rowdiv_i when rowdiv is not
// NULL), i < M, j < n, written column-major into C (ld ldc).  A: row-major
// (A(i, c) = A[i lda + c]) or column-major (A[c lda + i]); B: row-major
// (B[j ldb + c]).  amax_i >= max_c |A(i, c)| and bmax_j >= max_c |B(j, c)| for
// c < K.  Kmax bounds K (the tensor maps cover Kmax columns; values past K must
// be finite or zero in B).  With st != NULL the launch does nothing once
// st->done or st->m == 0; K = -1 means K = st->k and K = -2 means K = st->m; a
// nonzero c_koff moves C to C + st->k c_koff and writes only the first st->m
// of the n columns (the engine's new columns of F).
cudaError_t launch_ozgemm(const double* A, int64_t lda, bool a_colmajor, int64_t M, const double* amax,
                          const double* B, int64_t ldb, int n, const double* bmax, int K, int Kmax,
                          const FactorState* st, double* C, int64_t ldc, const double* rowdiv, int* flags,
                          cudaStream_t s, int64_t c_koff = 0);

// Products from seven-digit planes (ozmm.cu).  ozmm_map describes the planes of
// an R x ldk operand (plane s at planes + s plane, row i at + i ldk, K-major;
// ldk a multiple of 16, 16-byte aligned) for the A side (128-row boxes) or the
// B side (64-row boxes).  launch_ozmm: C(i, j) = sum_{c < K} A(i, c) B(j, c) for
// i < M, j < n into C (column-major, ld ldc); row exponents ea (or ea_const when
// ea is NULL) and eb likewise; columns of the planes past K up to a multiple of
// 16 must be zero.  With st != NULL nothing is done once st->done or st->m == 0;
// K = -1, -2, -3 mean st->k, st->m, st->kp; a nonzero c_koff moves C to
// C + st->k c_koff and writes the first st->m columns, and pout != NULL also
// receives their digit planes (exponent 1) at columns st->kp .. of an operand
// with row length pout_ld and plane size pout_plane (zeros up to st->kp plus
// st->m rounded up to 16; pout 16-byte aligned, pout_ld a multiple of 16,
// st->kp a multiple of 16).
// digits: 7 (FP64 operands) or 3 (FP32 operands: T = round(x 2^(22 - E)), the
// three pairs of levels 0-2); rowdiv != NULL divides row i of C by rowdiv[i].
bool ozmm_map(CUtensorMap* map, const uint16_t* planes, int64_t rows, int64_t ldk, int64_t plane, bool a_side,
              int digits = 7);
cudaError_t launch_ozmm(const CUtensorMap& ma, const CUtensorMap& mb, const int* ea, int ea_const, const int* eb,
                        int eb_const, int64_t M, int n, int K, const FactorState* st, double* C, int64_t ldc,
                        int64_t c_koff, uint16_t* pout, int64_t pout_ld, int64_t pout_plane, int* flags,
                        cudaStream_t s, int digits = 7, const double* rowdiv = nullptr);

}  // namespace kevd
