// Shared device helpers of libkevd (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/kevd.h"

#define KEVD_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return KEVD_ECUDA;             \
    } while (0)

#define KEVD_LAUNCH_CHECK()                                   \
    do {                                                      \
        if (cudaGetLastError() != cudaSuccess) return KEVD_ECUDA; \
    } while (0)

namespace kevd {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Bump allocator over the caller's workspace.  sizes are recorded with the
// same calls by the *_workspace functions, so the carve order is the layout.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count) {
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += align_up(count * sizeof(T));
        return p;
    }
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): multipliers
// 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
// Counter (draw j, round i, stream, 0); key = (seed lo, seed hi).  The uniform
// is ((w0 >> 5) * 2^26 + (w1 >> 6)) / 2^53, exact in double.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double philox_uniform(uint64_t seed, uint32_t stream, uint32_t rnd,
                                                 uint32_t j) {
    uint32_t c0 = j, c1 = rnd, c2 = stream, c3 = 0;
    uint32_t k0 = (uint32_t)(seed & 0xffffffffull), k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return ((double)(c0 >> 5) * 67108864.0 + (double)(c1 >> 6)) * (1.0 / 9007199254740992.0);
}

// Warp-level helpers ---------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (value, index) max with the lowest index winning ties.
__device__ __forceinline__ void argmax_merge(double& v, int64_t& i, double v2, int64_t i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

__device__ __forceinline__ void warp_argmax(double& v, int64_t& i) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
        argmax_merge(v, i, v2, i2);
    }
}

// Block sum in a fixed order (deterministic); all threads get the result.
// smem: at least 32 doubles.
__device__ inline double block_sum(double v, double* smem) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) smem[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? smem[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) smem[0] = t;
    __syncthreads();
    double r = smem[0];
    __syncthreads();
    return r;
}

// Upper-triangular tile index -> (I, J), I <= J, over nb x nb tiles (row-major
// over the upper triangle: t = 0 .. nb(nb+1)/2 - 1).
__device__ __forceinline__ void tri_decode(int t, int nb, int& I, int& J) {
    I = 0;
    int rowlen = nb;
    while (t >= rowlen) {
        t -= rowlen;
        ++I;
        --rowlen;
    }
    J = I + t;
}

}  // namespace kevd
