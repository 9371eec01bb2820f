// Householder reflector of one column in the zlarfg convention, in FP64 and in
// double-float (used by the tridiagonal reductions).
#pragma once

#include <cuda_runtime.h>

#include "dfloat.h"
#include "fp64_fast.h"

namespace bse {

// Reflector k from alpha = (column k)_{k+1} and sigma = sum_{r>k+1} |(column k)_r|^2
// in the zlarfg convention (v_{k+1} = 1): beta = -sign(Re alpha) sqrt(|alpha|^2 + sigma),
// tau = (beta - alpha) / beta, v_r = x_r / (alpha - beta).  FP64 version, for
// squared norms outside the safe range of the double-float one.
__device__ inline void reflector_fp64(double2 al, double sigma, double2& tau, double2& inv, double& beta) {
    if (sigma == 0.0 && al.y == 0.0) {
        tau = make_double2(0.0, 0.0);
        beta = al.x;
        inv = make_double2(0.0, 0.0);
        return;
    }
    const double nrm2 = fma(al.x, al.x, fma(al.y, al.y, sigma));
    const double y = copysign(rsqrt_nr(nrm2), al.x);   // -1/beta
    beta = -nrm2 * y;
    tau = make_double2(fma(al.x, y, 1.0), al.y * y);
    const double2 den = make_double2(al.x - beta, al.y);
    const double rm = rcp_nr(fma(den.x, den.x, den.y * den.y));
    inv = make_double2(den.x * rm, -den.y * rm);
}

// The same in double-float: a few hundred FP32 cycles instead of a chain of
// dependent FP64 instructions
__device__ inline void reflector(cdf al, float2 sigma, cdf& tau, cdf& inv, float2& beta) {
    if (sigma.x == 0.f && al.z == 0.f && al.w == 0.f) {
        tau = cdf_zero();
        beta = make_float2(al.x, al.y);
        inv = cdf_zero();
        return;
    }
    float s = sigma.x, lo = sigma.y;
    df_acc(s, lo, al.x, al.y, al.x, al.y);
    df_acc(s, lo, al.z, al.w, al.z, al.w);
    const float2 nrm2 = df_fin(s, lo);
    if (!(nrm2.x >= 0x1p-100f && nrm2.x <= 0x1p100f)) {
        double2 t, iv;
        double b;
        reflector_fp64(cdf_to(al), df_to(sigma), t, iv, b);
        tau = cdf_from(t);
        inv = cdf_from(iv);
        beta = df_from(b);
        return;
    }
    const float2 nrm = df_sqrt(nrm2);
    beta = al.x < 0.f ? nrm : df_neg(nrm);
    const float2 rb = df_rcp(beta);
    const float2 ar = df_mul(make_float2(al.x, al.y), rb), ai = df_mul(make_float2(al.z, al.w), rb);
    const float2 tr = df_add(make_float2(1.f, 0.f), df_neg(ar));
    tau = make_float4(tr.x, tr.y, -ai.x, -ai.y);
    const float2 dr = df_add(make_float2(al.x, al.y), df_neg(beta));
    const float2 di = make_float2(al.z, al.w);
    float q = 0.f, ql = 0.f;
    df_acc(q, ql, dr.x, dr.y, dr.x, dr.y);
    df_acc(q, ql, di.x, di.y, di.x, di.y);
    const float2 rm = df_rcp(df_fin(q, ql));
    const float2 ir = df_mul(dr, rm), ii = df_mul(di, rm);
    inv = make_float4(ir.x, ir.y, -ii.x, -ii.y);
}

}  // namespace bse
