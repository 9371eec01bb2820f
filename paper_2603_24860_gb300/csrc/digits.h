// Exact split of double-float values into balanced base-128 digits for the
// bf16 digit GEMMs on the tensor cores (her2k_tc.cu, zgemm_tc.cu).
#pragma once

#include <cuda_runtime.h>

#include "dfloat.h"

namespace bse {

constexpr int kDigits = 8;   // digits per value: 7 bits each below a leading 8-bit one (56 bits)

// x 2^p for a float x and |p| <= 250 (two exact power-of-two factors)
__device__ __forceinline__ float scale_pow2(float x, int p) {
    const int p1 = p / 2, p2 = p - p1;
    return (x * __int_as_float((127 + p1) << 23)) * __int_as_float((127 + p2) << 23);
}

// Balanced base-128 digits d_0 .. d_7 (weights 2^49 .. 2^0, stored pre-scaled by 2^-7k,
// so that each is exact in bf16) of rint(x 2^(56-e)) for a double-float x = h + l with
// |x| < 2^e, without FP64 or 64-bit integer arithmetic: (h, l) scaled by 2^(56-e), then per
// digit q = rint(h / w) for w = 2^(49-7k), h <- h - q w (exact: a multiple of ulp(h) of at
// most w/2 + |l|), and (h, l) renormalised by TwoSum; the last digit is rint(h + l).
// |d_0| <= 128 and |d_k| <= 64 (up to the size of l), so that a product of two digits is an
// integer below 2^14 and the sums of the digit GEMMs stay exact in FP32.
__device__ __forceinline__ void df_digits8(float h, float l, int e, float* d) {
    float hs = scale_pow2(h, 56 - e), ls = scale_pow2(l, 56 - e);
#pragma unroll
    for (int k = 0; k < kDigits - 1; ++k) {
        const float w = __int_as_float((127 + 49 - 7 * k) << 23), wi = __int_as_float((127 - 49 + 7 * k) << 23);
        const float q = rintf(hs * wi);
        hs = fmaf(-q, w, hs);
        two_sum(hs, ls, hs, ls);
        d[k] = q * __int_as_float((127 - 7 * k) << 23);
    }
    d[kDigits - 1] = rintf(hs + ls) * __int_as_float((127 - 7 * (kDigits - 1)) << 23);
}

// 2^e above every |h| of the given maximum (|h + l| < 2^e as well); 0 for a maximum of 0
__device__ __forceinline__ int exp_above_f(float m) { return m > 0.f ? ilogbf(m) + 1 : 0; }

}  // namespace bse
