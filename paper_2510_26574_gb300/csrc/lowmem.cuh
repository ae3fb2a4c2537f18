// The low-memory factor's lift, called by eig_topk_lowmem (eig.cu) after the
// r x r stage: U = D~^-1 F Y with F = K(:,S) W^-T rebuilt panel by panel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct KevdLowmemLift {
    const double* X;      // device, N x d row-major
    int d;
    double inv_eps;
    const int64_t* piv;   // device int64[rank]: the pivots S
    const double* W;      // device, rank x rank column-major (ld ldw): F(S,:)
    int64_t ldw;
    void* ws;             // device, kevd_lowmem_lift_bytes(N, d, rank) bytes, 256-byte aligned
};

size_t kevd_lowmem_lift_bytes(int64_t N, int d, int rank);

// Y (rank x k, ld = rank) is overwritten with W^-T Y.  Returns a KEVD_* status.
int kevd_lowmem_lift(const KevdLowmemLift& L, int64_t N, int rank, int k, double* Y, const double* dtil, double* U,
                     cudaStream_t s);
