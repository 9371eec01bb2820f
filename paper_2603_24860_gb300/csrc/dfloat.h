// Double-float arithmetic for sm_103a.
//
// A real number is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2: a 48-bit significand with FP32's exponent range.  On
// GB300 an SM retires 128 FP32 FMAs per clock but only 2 FP64 FMAs, so a
// double-float multiply-add of about a dozen FP32 instructions runs several
// times faster than the FP64 pipe.  The building blocks are the error-free
// transformations of floating-point arithmetic: Knuth's TwoSum (s + e = a + b
// exactly), Dekker's Fast2Sum (the same when |a| >= |b|), the FMA form of
// TwoProduct (p + e = a b exactly) and the Karp-Markstein correction of a
// square root.  Every operation is an _rn intrinsic, which the compiler
// neither contracts into an FMA nor reorders.
//
// Error model: additions are the "sloppy" kind (the low words are added
// without their own TwoSum), so a sum or product carries an error of a few
// units of 2^-48 relative to the magnitudes of its operands, the same form as
// the bound of an ordinary floating-point sum; the Householder reduction built
// on it is backward stable with unit roundoff about 2^-47.
#pragma once

#include <cuda_runtime.h>

namespace bse {

// complex double-float: real part (x, y), imaginary part (z, w)
using cdf = float4;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ float2 df_from(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ cdf cdf_from(double2 z) {
    const float2 r = df_from(z.x), i = df_from(z.y);
    return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ double2 cdf_to(cdf z) {
    return make_double2((double)z.x + (double)z.y, (double)z.z + (double)z.w);
}
__device__ __forceinline__ cdf cdf_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// (s, lo) += a b for double-floats a = (ah, al), b = (bh, bl): the rounded
// leading product enters s through TwoSum; its rounding error, TwoSum's error
// and the cross terms collect in lo (12 FP32 instructions)
__device__ __forceinline__ void df_acc(float& s, float& lo, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float pe = __fmaf_rn(ah, bh, -p);
    float t;
    two_sum(s, p, s, t);
    lo = __fadd_rn(lo, __fadd_rn(t, pe));
    lo = __fmaf_rn(ah, bl, lo);
    lo = __fmaf_rn(al, bh, lo);
}

// (s, lo) += a b for a float a and a double-float b = (bh, bl): a product with
// an exact FP32 factor needs one cross term (11 FP32 instructions)
__device__ __forceinline__ void df_acc1(float& s, float& lo, float a, float bh, float bl) {
    const float p = __fmul_rn(a, bh);
    const float pe = __fmaf_rn(a, bh, -p);
    float t;
    two_sum(s, p, s, t);
    lo = __fadd_rn(lo, __fadd_rn(t, pe));
    lo = __fmaf_rn(a, bl, lo);
}

// s + lo as a normalised double-float
__device__ __forceinline__ float2 df_fin(float s, float lo) {
    float h, l;
    fast_two_sum(s, lo, h, l);
    return make_float2(h, l);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    return df_fin(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return df_fin(p, e);
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// sqrt(a) for a > 0 normal: correctly rounded float root s0, then one
// Karp-Markstein step s0 + (a - s0^2) / (2 s0) with the residual formed exactly
__device__ __forceinline__ float2 df_sqrt(float2 a) {
    const float s0 = __fsqrt_rn(a.x);
    const float p = __fmul_rn(s0, s0);
    const float pe = __fmaf_rn(s0, s0, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), pe), a.y);   // a - s0^2, its leading bits
    return df_fin(s0, __fdiv_rn(r, __fmul_rn(2.f, s0)));
}

// 1/a for a normal and nonzero: correctly rounded float reciprocal r0, then
// one Newton step r0 + r0 (1 - a r0) with the residual formed exactly
__device__ __forceinline__ float2 df_rcp(float2 a) {
    const float r0 = __frcp_rn(a.x);
    const float p = __fmul_rn(a.x, r0);
    const float pe = __fmaf_rn(a.x, r0, -p);
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), pe), __fmul_rn(a.y, r0));   // 1 - a r0
    return df_fin(r0, __fmul_rn(r0, e));
}

__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) {
    const float2 r = df_add(make_float2(a.x, a.y), make_float2(b.x, b.y));
    const float2 i = df_add(make_float2(a.z, a.w), make_float2(b.z, b.w));
    return make_float4(r.x, r.y, i.x, i.y);
}

// a + b c
__device__ __forceinline__ cdf cdf_fma(cdf a, cdf b, cdf c) {
    float sr = a.x, lr = a.y, si = a.z, li = a.w;
    df_acc(sr, lr, b.x, b.y, c.x, c.y);
    df_acc(sr, lr, -b.z, -b.w, c.z, c.w);
    df_acc(si, li, b.x, b.y, c.z, c.w);
    df_acc(si, li, b.z, b.w, c.x, c.y);
    const float2 r = df_fin(sr, lr), i = df_fin(si, li);
    return make_float4(r.x, r.y, i.x, i.y);
}

__device__ __forceinline__ cdf cdf_mul(cdf b, cdf c) { return cdf_fma(cdf_zero(), b, c); }

// acc + conj(a) b
__device__ __forceinline__ cdf cdf_dot_acc(cdf acc, cdf a, cdf b) {
    float sr = acc.x, lr = acc.y, si = acc.z, li = acc.w;
    df_acc(sr, lr, a.x, a.y, b.x, b.y);
    df_acc(sr, lr, a.z, a.w, b.z, b.w);
    df_acc(si, li, a.x, a.y, b.z, b.w);
    df_acc(si, li, -a.z, -a.w, b.x, b.y);
    const float2 r = df_fin(sr, lr), i = df_fin(si, li);
    return make_float4(r.x, r.y, i.x, i.y);
}

// q - v conj(wc) - w conj(vc): one element of a Hermitian rank-2 update
__device__ __forceinline__ cdf cdf_rank2(cdf q, cdf v, cdf w, cdf wc, cdf vc) {
    float sr = q.x, lr = q.y, si = q.z, li = q.w;
    df_acc(sr, lr, -v.x, -v.y, wc.x, wc.y);
    df_acc(sr, lr, -v.z, -v.w, wc.z, wc.w);
    df_acc(sr, lr, -w.x, -w.y, vc.x, vc.y);
    df_acc(sr, lr, -w.z, -w.w, vc.z, vc.w);
    df_acc(si, li, -v.z, -v.w, wc.x, wc.y);
    df_acc(si, li, v.x, v.y, wc.z, wc.w);
    df_acc(si, li, -w.z, -w.w, vc.x, vc.y);
    df_acc(si, li, w.x, w.y, vc.z, vc.w);
    const float2 r = df_fin(sr, lr), i = df_fin(si, li);
    return make_float4(r.x, r.y, i.x, i.y);
}

__device__ __forceinline__ cdf cdf_shfl_xor(cdf v, int o) {
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o),
                       __shfl_xor_sync(0xffffffffu, v.z, o), __shfl_xor_sync(0xffffffffu, v.w, o));
}

__device__ __forceinline__ cdf cdf_warp_sum(cdf v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = cdf_add(v, cdf_shfl_xor(v, o));
    return v;
}

}  // namespace bse
