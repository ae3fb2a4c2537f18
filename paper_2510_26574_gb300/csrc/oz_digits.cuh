// Seven-digit Ozaki slicing of FP64 values for the tensor-core products of the
// FP64 path (ozgemm.cu, ozmm.cu and the plane producers of factor.cu).
#pragma once
#include <stdint.h>

namespace kevd {

constexpr int kDigits = 7;

// Seven digit planes of two values of one row (p_s = d_s 2^(-8 s) as BF16,
// packed two per word).  sh0 = 1021 + E: T = x 2^(54 - E) = m 2^(e - sh0) for
// x = m 2^(e - 1075), |T| < 2^54 (all 53 bits of x for |x| >= 2^(E - 1)).  The
// balanced digits are the bytes of T + 0x80808080808080 minus 128, and BF16 of
// d 2^(-8 s) is float(bits(M_s) + d) - M_s with M_s = 1.5 * 2^(23 - 8 s) (ulp
// 2^(-8 s)).  A row with E <= -900 gives zeros, as do subnormal, infinite or NaN
// values (they never meet a nonzero digit of the other factor).
__device__ __forceinline__ void digits2(double x0, double x1, int sh0, uint32_t (&w)[kDigits]) {
    unsigned long long U[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const double x = u ? x1 : x0;
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        const int e = (int)((b >> 52) & 0x7FF);
        const int sh = sh0 - e;                                   // >= -1 since |x| < 2^E
        long long T = 0;
        if (e != 0 && e != 0x7FF && sh < 62 && sh >= -1) {
            const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
            T = sh <= 0 ? (long long)(m << (-sh)) : (long long)(((m >> (sh - 1)) + 1) >> 1);
            T = T < 0x3FFFFFFFFFFFFFll ? T : 0x3FFFFFFFFFFFFFll;  // |x| rounding up to 2^E
            if ((long long)b < 0) T = -T;
        }
        U[u] = (unsigned long long)(T + 0x80808080808080ll);
    }
#pragma unroll
    for (int s = 0; s < kDigits; ++s) {
        const int bi = kDigits - 1 - s;
        const float Ms = 1.5f * __int_as_float((150 - 8 * s) << 23);
        const uint32_t mb = __float_as_uint(Ms) - 128u;
        const float f0 = __fsub_rn(__uint_as_float(mb + (uint32_t)((U[0] >> (8 * bi)) & 255u)), Ms);
        const float f1 = __fsub_rn(__uint_as_float(mb + (uint32_t)((U[1] >> (8 * bi)) & 255u)), Ms);
        w[s] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
    }
}

// TMEM accumulator of the digit pair (s, lv - s) of level lv.  Levels 0-3 and
// the two halves of level 4 ({s <= 2}, {s >= 3}) each sum integers on one grid
// (2^(-8 lv)) whose magnitude stays within 2^24 over a 256-column chunk, so
// their FP32 sums are exact; levels 5 and 6 share one inexact accumulator.  A
// merged level 4 would not do: the tensor core truncates a small addend to the
// accumulator's ulp, and the bias of ~2^-24 of the level-4 sum per MMA reaches
// 2^-48 of the product, well above FP64 rounding.
__device__ __forceinline__ constexpr int acc_of(int lv, int s) {
    return lv < 4 ? lv : lv == 4 ? (s <= 2 ? 4 : 5) : 6;
}

// Exponent E with mx < 2^E (frexp's) from the bits of mx >= 0, in integer
// arithmetic; E = -900 marks a zero (or negligible, below 2^-900) row.
__device__ __forceinline__ int exp_of(double mx) {
    const int be = (int)((unsigned long long)__double_as_longlong(mx) >> 52) & 0x7FF;
    return be >= 123 ? be - 1022 : -900;
}

// 2^e as a double for -1022 <= e <= 1023.
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// D-digit slicing (D <= 7) of a row with exponent E (max |row| < 2^E, E = -900
// for a zero row): T = round(x 2^(8 D - 2 - E)), |T| < 2^(8 D - 2), so that
// x = 2^(E - 6) sum_s d_s 2^(-8 s) for every D (the product scale 2^(E_a + E_b
// - 12) does not depend on D).  Zero, subnormal, infinite or NaN values give 0.
template <int D>
__device__ __forceinline__ long long oz_T_f64(double x, int E) {
    if (E <= -900) return 0;
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const int sh = 1077 - 8 * D + E - e;                      // >= -1 since |x| < 2^E
    long long T = 0;
    if (e != 0 && e != 0x7FF && sh < 62 && sh >= -1) {
        const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        T = sh <= 0 ? (long long)(m << (-sh)) : (long long)(((m >> (sh - 1)) + 1) >> 1);
        const long long lim = (1ll << (8 * D - 2)) - 1;
        T = T < lim ? T : lim;
        if ((long long)b < 0) T = -T;
    }
    return T;
}

template <int D>
__device__ __forceinline__ long long oz_T_f32(float x, int E) {
    if (E <= -900) return 0;
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFF);
    const int sh = 152 - 8 * D + E - e;                       // x = m 2^(e - 150), m < 2^24
    long long T = 0;
    if (e != 0 && e != 0xFF && sh < 30 && sh >= -40) {
        const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
        T = sh <= 0 ? (long long)(m << (-sh)) : (long long)(((m >> (sh - 1)) + 1) >> 1);
        const long long lim = (1ll << (8 * D - 2)) - 1;
        T = T < lim ? T : lim;
        if (b >> 31) T = -T;
    }
    return T;
}

// The D planes of two sliced values (p_s = d_s 2^(-8 s) as BF16, packed two per
// word, plane s in w[s]): the balanced digits are the bytes of T + 0x80..80.
template <int D>
__device__ __forceinline__ void oz_planes2(long long T0, long long T1, uint32_t (&w)[D]) {
    unsigned long long off = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) off |= 0x80ull << (8 * i);
    const unsigned long long U0 = (unsigned long long)T0 + off, U1 = (unsigned long long)T1 + off;
#pragma unroll
    for (int s = 0; s < D; ++s) {
        const int bi = D - 1 - s;
        const float Ms = 1.5f * __int_as_float((150 - 8 * s) << 23);
        const uint32_t mb = __float_as_uint(Ms) - 128u;
        const float f0 = __fsub_rn(__uint_as_float(mb + (uint32_t)((U0 >> (8 * bi)) & 255u)), Ms);
        const float f1 = __fsub_rn(__uint_as_float(mb + (uint32_t)((U1 >> (8 * bi)) & 255u)), Ms);
        w[s] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
    }
}

// Plane s alone of two sliced values (the word oz_planes2 puts in w[s]).
template <int D>
__device__ __forceinline__ uint32_t oz_word(long long T0, long long T1, int s) {
    unsigned long long off = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) off |= 0x80ull << (8 * i);
    const int bi = D - 1 - s;
    const float Ms = 1.5f * __int_as_float((150 - 8 * s) << 23);
    const uint32_t mb = __float_as_uint(Ms) - 128u;
    const float f0 = __fsub_rn(__uint_as_float(mb + (uint32_t)((((unsigned long long)T0 + off) >> (8 * bi)) & 255u)), Ms);
    const float f1 = __fsub_rn(__uint_as_float(mb + (uint32_t)((((unsigned long long)T1 + off) >> (8 * bi)) & 255u)), Ms);
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
}

// Digit planes of two values x0, x1 on a row with exponent E (max |row| < 2^E,
// E = -900 for a zero row).
__device__ __forceinline__ void digits2_e(double x0, double x1, int E, uint32_t (&w)[kDigits]) {
    digits2(x0, x1, E > -900 ? 1021 + E : 4096, w);
}

}  // namespace kevd
