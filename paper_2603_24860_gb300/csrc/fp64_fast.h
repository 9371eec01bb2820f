// FP64 helpers for GB300, whose FP64 pipe runs two lanes per clock per SM:
// an IEEE divide there costs hundreds of cycles of FP64 issue, so hot loops
// use a Newton-Raphson reciprocal instead.
#pragma once

#include <cuda_runtime.h>

namespace bse {

// 2^e for -1022 <= e <= 1023, exactly
__device__ __forceinline__ double exp2i(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// 1/a by Newton-Raphson (y <- y + y (1 - a y), quadratic convergence) from a
// single-precision seed of the mantissa: two steps take 23 bits past 53.  For
// normal, finite a; the result is within a few ulp of 1/a (not correctly
// rounded).
__device__ __forceinline__ double rcp_nr(double a) {
    const long long bits = __double_as_longlong(a);
    const int ex = (int)((bits >> 52) & 0x7ff) - 1023;
    const double m = __longlong_as_double((bits & 0x000fffffffffffffll) | 0x3ff0000000000000ll);   // [1, 2)
    double y = (double)__frcp_rn((float)m) * exp2i(-ex);
    y = copysign(y, a);
    double r = fma(-a, y, 1.0);
    y = fma(y, r, y);
    r = fma(-a, y, 1.0);
    y = fma(y, r, y);
    return y;
}

// 1/sqrt(a) by Newton-Raphson (y <- y (3 - a y^2) / 2, quadratic convergence)
// from a single-precision seed of a scaled into [1, 4): three steps take 23
// bits past 53 with margin.  For normal, finite a > 0; within a few ulp.
__device__ __forceinline__ double rsqrt_nr(double a) {
    const long long bits = __double_as_longlong(a);
    const int ex = (int)((bits >> 52) & 0x7ff) - 1023;
    const int h = ex >> 1;                                       // a = m 2^(2h), m in [1, 4)
    const double m = __longlong_as_double((bits & 0x000fffffffffffffll) |
                                          ((long long)(1023 + (ex - 2 * h)) << 52));
    double y = (double)rsqrtf((float)m);
    const double hm = 0.5 * m;
#pragma unroll
    for (int i = 0; i < 3; ++i) y = y * fma(-hm, y * y, 1.5);
    return y * exp2i(-h);
}

// sign bit of x (no FP64 compare: the FP64 pipe is the scarce unit)
__device__ __forceinline__ bool neg_bit(double x) { return __double_as_longlong(x) < 0; }

}  // namespace bse
