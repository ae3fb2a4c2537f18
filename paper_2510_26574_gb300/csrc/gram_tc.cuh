// Tensor-core (tcgen05) weighted Grams of an FP32 factor; see gram_tc.cu.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kevd {

// True when F can be read by the tensor map (16-byte aligned, ldf a multiple
// of 4, N < 2^31) and KEVD_GRAM=ffma does not ask for the FFMA kernel.
bool gram_tc_eligible(const float* F, int64_t ldf, int64_t N, int rank);

// Rows per split (a multiple of 64) and the split count for ntri tile pairs.
int64_t gram_tc_per(int64_t N, int64_t ntri, int nsm, int* nsplit);

// Column maxima, magic numbers and the Gram kernel: gpart receives
// nsplit x ntri x 2 x 128 x 128 FP32 partials (A, then C) for the FP64 split
// reduction.  wa, wc: FP32 weights zero-padded to a multiple of 64 rows (wc
// NULL: the first Gram only); cmax, mag: 3 x rank scratch; flags bit 2 is set
// if a bounded wait gave up.
cudaError_t launch_gram_tc(const float* F, int64_t ldf, int64_t N, int rank, const float* wa, const float* wc,
                           unsigned* cmax, float* mag, float* gpart, int* flags, int nb, int ntri, int64_t per,
                           int nsplit, cudaStream_t s);

// FP64 factor: weighted Grams on the tensor cores at FP64 accuracy (gram_oz.cu).
// wa, wc: FP64 weights zero-padded to a multiple of 64 rows (wc NULL: A only);
// cmax: 3 x rank, Ecol: 3 x rank scratch; gpart: gram_oz_partial_doubles(...);
// planes: gram_oz_plane_bytes(...) bytes, 16-byte aligned (the digit planes of
// one slab of rows).  Writes A (and C) in full, exactly symmetric.
bool gram_oz_eligible(const double* F, int64_t ldf, int64_t N, int rank);
size_t gram_oz_partial_doubles(int64_t N, int rank, int ngram, int nsm);
size_t gram_oz_plane_bytes(int64_t N, int rank, int ngram);
// wa_rz, wc_rz: N floats of scratch each (the weights' truncated FP32 copies for
// the column bounds; wc_rz unused when wc is NULL).
cudaError_t launch_gram_oz(const double* F, int64_t ldf, int64_t N, int rank, const double* wa, const double* wc,
                           float* wa_rz, float* wc_rz, unsigned long long* cmax, int* Ecol, double* gpart,
                           uint16_t* planes, int* flags, double* A, double* C, int nsm, cudaStream_t s);

}  // namespace kevd
