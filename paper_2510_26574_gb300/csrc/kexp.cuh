// exp(t) for t <= 0 at FP64 accuracy with four FP64 operations, for the
// Gaussian kernel values of the FP64 engine on the tensor cores (FP64 is the
// slow pipe of this GPU; the integer pipe is not).  Tang's table-driven method
// (P. T. P. Tang, ACM TOMS 15(2), 1989) with 2^10 table points and the
// polynomial in 64-bit fixed point:
//   n = rint(t 2^10 / ln 2), r = t - n ln 2 / 2^10 (two-part constant, |r| <= ln 2 / 2^11),
//   exp(t) = 2^(n >> 10) 2^((n & 1023) / 2^10) (1 + r + r^2/2 + r^3/6 + r^4/24),
// the omitted terms below 2^-64; the table holds round(2^(j / 2^10) 2^62), r is
// taken to Q62 and every product to Q62 by truncation (errors of a few 2^-62),
// and the result is rounded once to 53 bits: within one ulp of exp(t).  The
// split of ln 2 / 2^10 into C1 (29 significant bits, so that n C1 is exact for
// |n| < 2^24) and C2 was computed from ln 2 to 60 digits.  For t <= -708 the
// result is flushed to 0 (exp(-708) < 2^-1021, far below every use).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kevd {

// The table round(2^(j / 1024) 2^62), j < 1024, on the current device (filled
// once per process and device from host long double arithmetic): its device
// address in *tbl.
cudaError_t kexp_table(cudaStream_t s, const unsigned long long** tbl);

__device__ __forceinline__ long long kexp_mulq62(long long a, long long b) {   // (a b) >> 62, signed
    const unsigned long long hi = (unsigned long long)__mul64hi(a, b);
    const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
    return (long long)((hi << 2) | (lo >> 62));
}

// tbl: the 1024-entry table (shared or global memory).
__device__ __forceinline__ double kexp(double t, const unsigned long long* tbl) {
    if (!(t > -708.0)) return 0.0;
    const double tt = fma(t, 0x1.71547652b82fep+10, 0x1.8p52);    // 1.5 2^52 + rint(t 2^10 / ln 2)
    const int n = (int)(__double_as_longlong(tt) - __double_as_longlong(0x1.8p52));
    const double nd = tt - 0x1.8p52;
    double r = fma(-nd, 0x1.62e42ffp-11, t);
    r = fma(-nd, -0x1.718432a1b0e26p-45, r);
    // r to Q62 (|r| < 2^-11: a right shift of the 53-bit significand)
    const long long rb = __double_as_longlong(r);
    const int re = (int)((rb >> 52) & 0x7FF);
    long long R = 0;
    const int sh = 1013 - re;
    if (re != 0 && sh >= 0 && sh < 64) {
        const unsigned long long m = ((unsigned long long)rb & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        R = (long long)(m >> sh);
        if (rb < 0) R = -R;
    }
    long long a = 192153584101141163ll;                  // 2^62 / 24
    a = 768614336404564651ll + kexp_mulq62(R, a);        // 2^62 / 6
    a = 2305843009213693952ll + kexp_mulq62(R, a);       // 2^62 / 2
    a = 4611686018427387904ll + kexp_mulq62(R, a);       // 2^62
    const unsigned long long p = (unsigned long long)(4611686018427387904ll + kexp_mulq62(R, a));
    const unsigned long long T = tbl[n & 1023];
    unsigned long long M = (__umul64hi(T, p) << 2) | ((T * p) >> 62);   // 2^(j/1024) p(r) 2^62
    int q = n >> 10;
    if (M < (1ull << 62)) {
        M <<= 1;
        --q;
    }
    unsigned long long mant = (M + (1ull << 9)) >> 10;
    if (mant >> 53) {
        mant >>= 1;
        ++q;
    }
    return __longlong_as_double((long long)(((unsigned long long)(q + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace kevd
