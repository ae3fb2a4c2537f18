// FP64-accurate tensor-core products C = A B^T along rows (ozgemm.cu).
#pragma once
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

}  // namespace kevd
