// Status strings, option defaults and workspace sizing of the libkevd C-ABI.
#include "common.cuh"

size_t kevd_factor_ws(int64_t N, int32_t d, int32_t r, const kevd_opts* o);
size_t kevd_normalize_ws(int64_t N, int32_t rank, bool fp64);
size_t kevd_eig_ws(int64_t N, int32_t r, int32_t k);
size_t kevd_fix_ws(int64_t N, int32_t k);
size_t kevd_lowmem_factor_ws(int64_t N, int32_t d, int32_t r, const kevd_opts* o);
size_t kevd_lowmem_normalize_ws(int64_t N, int32_t d, int32_t rank);
size_t kevd_lowmem_eig_ws(int64_t N, int32_t d, int32_t r, int32_t k);

extern "C" size_t kevd_workspace_bytes(int which, int64_t N, int32_t d, int32_t r, int32_t k,
                                       const kevd_opts* opts) {
    switch (which) {
        case KEVD_WS_FACTOR: return kevd_factor_ws(N, d, r, opts);
        case KEVD_WS_NORMALIZE:   // opts->precision = KEVD_PREC_BF16X3: an FP32 factor (no digit planes)
            return r <= N ? kevd_normalize_ws(N, r, !(opts && opts->precision == KEVD_PREC_BF16X3)) : 0;
        case KEVD_WS_EIG: return r <= N ? kevd_eig_ws(N, r, k) : 0;
        case KEVD_WS_FIX: return kevd_fix_ws(N, k);
        case KEVD_WS_LOWMEM_FACTOR: return kevd_lowmem_factor_ws(N, d, r, opts);
        case KEVD_WS_LOWMEM_NORMALIZE: return kevd_lowmem_normalize_ws(N, d, r);
        case KEVD_WS_LOWMEM_EIG: return r <= N ? kevd_lowmem_eig_ws(N, d, r, k) : 0;
        default: return 0;
    }
}

extern "C" const char* kevd_status_string(int status) {
    switch (status) {
        case KEVD_OK: return "ok";
        case KEVD_EINVAL: return "invalid argument or non-finite input";
        case KEVD_ED_NONPOS: return "degree vector d~ = F F^T 1 has a non-positive entry";
        case KEVD_EQ_NONPOS: return "degree vector q~ = F F^T d~^-1 has a non-positive entry";
        case KEVD_ECUDA: return "CUDA runtime or cuSOLVER error";
        case KEVD_EWORKSPACE: return "workspace missing, misaligned or too small";
        case KEVD_ETIMEOUT: return "a bounded device-side wait gave up";
        case KEVD_EEIG: return "symmetric eigensolver did not converge";
        case KEVD_ESCRATCH: return "problem exceeds the static scratch of rpchol_factor_noalloc (16 MiB)";
        default: return "unknown status";
    }
}

extern "C" void kevd_opts_init(kevd_opts* o, int32_t precision) {
    if (!o) return;
    o->mode = KEVD_ARPC;
    o->precision = precision;
    o->block_b = 64;
    o->until_rank = 0;
    o->max_rounds = 0;
    o->reserved = 0;
    o->seed = 0;
    // FP32 factors: stop at sum(rho) <= 1e-6 N, the resolution of FP32 kernel
    // values, so that pivots whose residuals are rounding noise stay out of F
    o->tol = precision == KEVD_PREC_BF16X3 ? 1e-6 : 0.0;
}
