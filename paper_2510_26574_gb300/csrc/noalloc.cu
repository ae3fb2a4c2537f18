// rpchol_factor_noalloc: rpchol_factor for callers that cannot allocate device
// memory.  The workspace is a file-scope device array of fixed size that every
// GPU which loads this library holds until the process exits.
#include "common.cuh"

size_t kevd_factor_ws_mode(int64_t N, int32_t d, int32_t r, const kevd_opts* o, bool allow_oz);
int rpchol_factor_impl(const void* X, int x_dtype, int64_t N, int32_t d, double eps, int32_t r,
                       const kevd_opts* opts, void* F, int f_dtype, int64_t ldf, int64_t* pivots, double* rho,
                       int64_t* proposals, kevd_factor_info* info, void* workspace, size_t ws_bytes, void* stream,
                       bool allow_oz);

namespace {

// The scratch itself.  Host code must not use the symbol as an address: on the
// host it only names a stand-in, so its device address is looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KEVD_NOALLOC_SCRATCH_BYTES];

}  // namespace

extern "C" int rpchol_factor_noalloc(const void* X, int x_dtype, int64_t N, int32_t d, double eps, int32_t r,
                                     const kevd_opts* opts, void* F, int f_dtype, int64_t ldf, int64_t* pivots,
                                     double* rho, int64_t* proposals, kevd_factor_info* info, void* stream) {
    // the FP64 engine here keeps its products on the FP64 pipe: the tensor-core
    // form's two N x b product arrays would not fit the static array
    const size_t need = kevd_factor_ws_mode(N, d, r, opts, false);
    if (need > (size_t)KEVD_NOALLOC_SCRATCH_BYTES) return KEVD_ESCRATCH;
    // The array's device address, looked up on every call with the caller's
    // device current: it is cheap, allocates nothing, and stays right if the
    // context was reset or replaced since an earlier call (a cached address
    // would then point at memory the array no longer occupies).
    void* scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch) return KEVD_ECUDA;
    // Every buffer the factorisation reads from the workspace is written by it
    // first (its set-up kernel zeroes the round state), so the contents left by
    // an earlier call need no clearing here.
    return rpchol_factor_impl(X, x_dtype, N, d, eps, r, opts, F, f_dtype, ldf, pivots, rho, proposals, info, scratch,
                              (size_t)KEVD_NOALLOC_SCRATCH_BYTES, stream, false);
}
