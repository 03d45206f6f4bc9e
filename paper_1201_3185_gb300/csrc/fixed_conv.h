// Conversions between IEEE-754 binary64 and int64 on the integer pipe, for
// the once-per-solve kernels of the fixed-point defect correction.  On this
// GPU the FP64 conversion instructions run at a few operations per clock per
// SM; these functions decode the binary64 fields (sign, 11-bit biased
// exponent, 52-bit fraction) and round to nearest, ties to even, as the
// standard defines, with 64-bit integer shifts and adds only.  Plain C++: the
// host compiler builds the same code for the tests that pin them.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define QUMOND_HD __host__ __device__ __forceinline__
#else
#define QUMOND_HD inline
#endif

namespace qumond {

QUMOND_HD long long f64_bits(double x)
{
    long long b;
    memcpy(&b, &x, sizeof b);
    return b;
}

QUMOND_HD double f64_from_bits(long long b)
{
    double x;
    memcpy(&x, &b, sizeof x);
    return x;
}

// round(x) to the nearest integer, ties to even, for |x| < 2^63; larger
// magnitudes (and infinities, NaN) saturate to +-2^62, which only a diverging
// solve reaches.
QUMOND_HD long long f64_to_i64_rn(double x)
{
    const long long b = f64_bits(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex < 1022) return 0;  // |x| < 1/2 (zero and subnormals included) rounds to 0
    const int sh = 1075 - ex;
    if (sh < -10) return b < 0 ? -(1LL << 62) : (1LL << 62);
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);  // significand: x = m 2^(ex - 1075)
    long long q;
    if (sh <= 0) {
        q = m << (-sh);  // an integer already
    } else {
        q = m >> sh;
        const long long rem = m & ((1LL << sh) - 1), half = 1LL << (sh - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
    }
    return b < 0 ? -q : q;
}

// v as the nearest binary64 value, ties to even, times 2^e (exact scaling by a
// power of two: the caller keeps the result a normal number), for |v| < 2^63.
QUMOND_HD double i64_to_f64_rn_scaled(long long v, int e)
{
    if (v == 0) return 0.0;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
#if defined(__CUDA_ARCH__)
    const int top = 63 - __clzll((long long)a);  // index of the leading one bit
#else
    const int top = 63 - __builtin_clzll(a);
#endif
    unsigned long long m;  // 53-bit significand
    int ex = top;          // value = m 2^(ex - 52)
    if (top <= 52) {
        m = a << (52 - top);
    } else {
        const int sh = top - 52;
        m = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            ++m;
            if (m == (1ull << 53)) {  // the rounding carried into a new leading bit
                m >>= 1;
                ++ex;
            }
        }
    }
    const long long bits = (long long)(((unsigned long long)(v < 0) << 63) |
                                       ((unsigned long long)(ex + e + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull));
    return f64_from_bits(bits);
}

}  // namespace qumond
