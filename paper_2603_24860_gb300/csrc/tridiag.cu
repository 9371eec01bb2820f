// Levels and oscillator strengths of a Hermitian block without eigenvectors
// (sm_103a).
//
// Eqs. oscillator and oscillatorA need, for every eigenpair (Omega_l, a_l) of
// a block H, the weight |a_l^T b|^2 with b = U^T B.  With c = conj(b) this is
// |<c, a_l>|^2: the weights of the spectral measure of H seen from c.  A
// reflector H0 maps c to a multiple of e_0; the Householder reduction
// Q^H (H0 H H0) Q = T, whose reflectors act on rows 1..n-1 only, keeps e_0
// fixed, so the weights are ||c||^2 z_0(l)^2 with z(l) the eigenvectors of the
// real symmetric tridiagonal T (the Gauss quadrature of that measure).  The
// levels come from Sturm-count bisection of T, the first components from a
// twisted factorisation of T - Omega_l, O(n) per level; no eigenvector matrix
// is formed or back-transformed.
//
// GB300 layout: the reduction is one persistent cooperative kernel with one
// CTA per SM.  Column j of the block belongs to CTA j mod G; for n up to
// about 1400 every CTA keeps its columns in shared memory for the whole
// reduction (152 x 227 KB hold a 1400 x 1400 complex matrix), otherwise they
// stay in global memory.  Because the block is Hermitian, (A v)_j is a dot
// product with column j, so each step needs no cross-CTA reduction except one
// scalar, and two grid barriers per step order the reflector and x = tau A v.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "fp64_fast.h"
#include "grid_sync.h"
#include "internal.h"

namespace bse {

namespace {

constexpr int kTriThreads = 256;
constexpr int kTriWarps = kTriThreads / 32;
constexpr int kChunk = 8;                 // columns reduced together

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rank-2 update  A_rc -= v_r conj(w_c) + w_r conj(v_c)  of a chunk, eight FMAs per element
template <int NC>
__device__ __forceinline__ void chunk_update(double2* cb, size_t cs, const double2* V, const double2* W,
                                             const int* jcol, int r0, int n) {
    double2 vj[NC], wj[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        vj[c] = V[jcol[c]];
        wj[c] = W[jcol[c]];
    }
    for (int r = r0 + (int)threadIdx.x; r < n; r += kTriThreads) {
        const double2 v = V[r], w = W[r];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double2 q = cb[c * cs + r];
            q.x = fma(-v.x, wj[c].x, q.x);
            q.x = fma(-v.y, wj[c].y, q.x);
            q.x = fma(-w.x, vj[c].x, q.x);
            q.x = fma(-w.y, vj[c].y, q.x);
            q.y = fma(-v.y, wj[c].x, q.y);
            q.y = fma(v.x, wj[c].y, q.y);
            q.y = fma(-w.y, vj[c].x, q.y);
            q.y = fma(w.x, vj[c].y, q.y);
            cb[c * cs + r] = q;
        }
    }
}

#define BSE_NC_DISPATCH(nc, F, ...)         \
    switch (nc) {                            \
        case 1: F<1>(__VA_ARGS__); break;    \
        case 2: F<2>(__VA_ARGS__); break;    \
        case 3: F<3>(__VA_ARGS__); break;    \
        case 4: F<4>(__VA_ARGS__); break;    \
        case 5: F<5>(__VA_ARGS__); break;    \
        case 6: F<6>(__VA_ARGS__); break;    \
        case 7: F<7>(__VA_ARGS__); break;    \
        default: F<8>(__VA_ARGS__); break;   \
    }

struct TriArgs {
    double2* A;           // n x n column-major, leading dimension n (updated in place in the global variant)
    int64_t n;
    const double2* v0;    // initial reflector
    const double* beta0;  // its (real) scalar
    double2* ncol;        // [2][n] the next column to be reflected, published by its owner, by parity
    double2* xbuf;        // [2][n] x = tau A v, by step parity
    double2* spart;       // [2][G] per-CTA parts of x^H v, by step parity
    double* d;            // [n] diagonal of T
    double* e;            // [n] off-diagonal of T (e[n-1] unused)
    unsigned* bar;        // barrier counter, zero on entry
    int* err;             // error flag, zero on entry
};

// One grid barrier per reflection step s (H(s) = I - tau v v^H on rows >= s+1,
// s = -1 being the start reflector H0 on all rows):
//   P1  x(s) and the parts of x^H v from all CTAs: alpha = -tau (x^H v)/2,
//       w = x + alpha v (shared memory)
//   P2  own columns j > s:  A_rj -= v_r conj(w_j) + w_r conj(v_j),  r > s
//   P3  every CTA applies the same update to the published copy of column
//       k = s+1 and forms reflector k from it (zlarfg convention, v_{k+1} = 1)
//   P4  the owner of column k+1 publishes it (its state before step k)
//   P5  x(k)_j = tau(k) sum_r conj(A_rj) v_r for own columns j > k (Hermitian:
//       (A v)_j is a column dot product) and this CTA's part of x^H v
//   grid barrier
template <bool kSmem>
__global__ void __launch_bounds__(kTriThreads, 1) tridiag_kernel(TriArgs a) {
    extern __shared__ __align__(16) double2 s_dyn[];
    __shared__ double2 s_s[kTriWarps];
    __shared__ double2 s_scal[2];   // [0] inv(alpha - beta) of the new reflector, [1] alpha of P1
    __shared__ double2 s_tau;
    __shared__ double s_sig[kTriWarps];
    __shared__ int s_flag;

    const int n = (int)a.n;
    const int G = gridDim.x, blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ncl = blk < n ? (n - 1 - blk) / G + 1 : 0;
    double2* V = s_dyn;
    double2* W = s_dyn + n;
    double2* C = s_dyn + 2 * (size_t)n;
    double2* s_cols = s_dyn + 3 * (size_t)n;
    auto col = [&](int l) -> double2* {
        return kSmem ? s_cols + (size_t)l * n : a.A + (size_t)(blk + l * G) * n;
    };
    const size_t cstride = kSmem ? (size_t)n : (size_t)G * n;
    if (kSmem)
        for (int l = 0; l < ncl; ++l) {
            const double2* src = a.A + (size_t)(blk + l * G) * n;
            for (int r = tid; r < n; r += kTriThreads) s_cols[(size_t)l * n + r] = src[r];
        }
    for (int r = tid; r < n; r += kTriThreads) V[r] = __ldcg(a.v0 + r);
    if (tid == 0) s_tau = make_double2(__ldcg(a.beta0), 0.0);
    __syncthreads();
    // column 0 as it is before the start reflector
    if (blk == 0)
        for (int r = tid; r < n; r += kTriThreads) a.ncol[r] = col(0)[r];
    unsigned nbar = 0;

    // P5 for reflector k (rows > k; k = -1: all rows): one warp per column, so
    // the only cross-lane FP64 work is one shuffle reduction per column
    auto dots = [&](int k) {
        const int r0 = k + 1;
        const double2 tau = s_tau;
        const int l0 = blk >= r0 ? 0 : (r0 - blk + G - 1) / G;
        double2* xb = a.xbuf + (size_t)(k & 1) * n;
        double2 sw = make_double2(0.0, 0.0);
        for (int l = l0 + wid; l < ncl; l += kTriWarps) {
            const double2* cl = col(l);
            double2 acc = make_double2(0.0, 0.0), acc2 = make_double2(0.0, 0.0);
            int r = r0 + lane;
            for (; r + 32 < n; r += 64) {
                const double2 a0 = cl[r], v0 = V[r], a1 = cl[r + 32], v1 = V[r + 32];
                acc.x = fma(a0.x, v0.x, acc.x);
                acc.x = fma(a0.y, v0.y, acc.x);
                acc.y = fma(a0.x, v0.y, acc.y);
                acc.y = fma(-a0.y, v0.x, acc.y);
                acc2.x = fma(a1.x, v1.x, acc2.x);
                acc2.x = fma(a1.y, v1.y, acc2.x);
                acc2.y = fma(a1.x, v1.y, acc2.y);
                acc2.y = fma(-a1.y, v1.x, acc2.y);
            }
            if (r < n) {
                const double2 a0 = cl[r], v0 = V[r];
                acc.x = fma(a0.x, v0.x, acc.x);
                acc.x = fma(a0.y, v0.y, acc.x);
                acc.y = fma(a0.x, v0.y, acc.y);
                acc.y = fma(-a0.y, v0.x, acc.y);
            }
            const double sx = warp_sum(acc.x + acc2.x), sy = warp_sum(acc.y + acc2.y);
            if (lane == 0) {
                const int j = blk + l * G;
                const double2 x = cmul(tau, make_double2(sx, sy));
                xb[j] = x;
                const double2 t = cmulc(x, V[j]);
                sw.x += t.x;
                sw.y += t.y;
            }
        }
        if (lane == 0) s_s[wid] = sw;
        __syncthreads();
        if (tid == 0) {
            double2 sp = make_double2(0.0, 0.0);
            for (int w = 0; w < kTriWarps; ++w) {
                sp.x += s_s[w].x;
                sp.y += s_s[w].y;
            }
            a.spart[(size_t)(k & 1) * G + blk] = sp;
        }
    };

    dots(-1);
    if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag)) return;

    for (int s = -1; s <= n - 2; ++s) {
        const int r0 = s + 1;
        const int k = s + 1;   // column reflected next
        const bool more = s < n - 2;
        // P1: gather x(s), the parts of x^H v and the published column k in one round trip
        const double2* xb = a.xbuf + (size_t)(s & 1) * n;
        const double2* nc_src = a.ncol + (size_t)(k & 1) * n;
        for (int r = r0 + tid; r < n; r += kTriThreads) {
            W[r] = __ldcg(xb + r);
            if (more) C[r] = __ldcg(nc_src + r);
        }
        if (wid == 0) {
            double sx = 0.0, sy = 0.0;
            const double2* sp = a.spart + (size_t)(s & 1) * G;
#pragma unroll 4
            for (int b = lane; b < G; b += 32) {
                const double2 p = __ldcg(sp + b);
                sx += p.x;
                sy += p.y;
            }
            sx = warp_sum(sx);
            sy = warp_sum(sy);
            if (lane == 0) {
                const double2 al = cmul(s_tau, make_double2(sx, sy));
                s_scal[1] = make_double2(-0.5 * al.x, -0.5 * al.y);
            }
        }
        __syncthreads();
        const double2 alpha = s_scal[1];
        for (int r = r0 + tid; r < n; r += kTriThreads) {
            const double2 v = V[r];
            double2 x = W[r];
            x.x = fma(alpha.x, v.x, fma(-alpha.y, v.y, x.x));
            x.y = fma(alpha.x, v.y, fma(alpha.y, v.x, x.y));
            W[r] = x;
        }
        __syncthreads();
        // P2: rank-2 update of own columns j >= r0
        const int l0 = blk >= r0 ? 0 : (r0 - blk + G - 1) / G;
        for (int c0 = l0; c0 < ncl; c0 += kChunk) {
            const int nc = min(kChunk, ncl - c0);
            int jcol[kChunk];
#pragma unroll
            for (int c = 0; c < kChunk; ++c) jcol[c] = blk + (c0 + c) * G;
            BSE_NC_DISPATCH(nc, chunk_update, col(c0), cstride, V, W, jcol, r0, n)
        }
        if (!more) break;
        // P3: column k after this step's update, then its reflector
        const double2 vk = V[k], wk = W[k];
        __syncthreads();
        double sg = 0.0;
        for (int r = k + tid; r < n; r += kTriThreads) {
            const double2 c = C[r], v = V[r], w = W[r];
            double2 cr;   // c - v conj(w_k) - w conj(v_k)
            cr.x = fma(-v.x, wk.x, fma(-v.y, wk.y, fma(-w.x, vk.x, fma(-w.y, vk.y, c.x))));
            cr.y = fma(-v.y, wk.x, fma(v.x, wk.y, fma(-w.y, vk.x, fma(w.x, vk.y, c.y))));
            W[r] = cr;
            if (r >= k + 2) sg = fma(cr.x, cr.x, fma(cr.y, cr.y, sg));
        }
        sg = warp_sum(sg);
        if (lane == 0) s_sig[wid] = sg;
        __syncthreads();
        if (tid == 0) {
            double sigma = 0.0;
            for (int w = 0; w < kTriWarps; ++w) sigma += s_sig[w];
            const double2 al = W[k + 1];
            double2 tau, inv;
            double beta;
            if (sigma == 0.0 && al.y == 0.0) {
                tau = make_double2(0.0, 0.0);
                beta = al.x;
                inv = make_double2(0.0, 0.0);
            } else {
                const double nrm2 = fma(al.x, al.x, fma(al.y, al.y, sigma));
                const double y = copysign(rsqrt_nr(nrm2), al.x);   // -1/beta
                beta = -nrm2 * y;
                tau = make_double2(fma(al.x, y, 1.0), al.y * y);     // (beta - alpha) / beta
                const double2 den = make_double2(al.x - beta, al.y);
                const double rm = rcp_nr(fma(den.x, den.x, den.y * den.y));
                inv = make_double2(den.x * rm, -den.y * rm);
            }
            s_scal[0] = inv;
            s_tau = tau;
            if (blk == 0) {
                a.d[k] = W[k].x;
                a.e[k] = beta;
            }
        }
        __syncthreads();
        {
            const double2 inv = s_scal[0];
            for (int r = k + 1 + tid; r < n; r += kTriThreads) V[r] = r == k + 1 ? make_double2(1.0, 0.0) : cmul(W[r], inv);
        }
        __syncthreads();
        // P4: publish column k+1 (state before step k)
        if (k + 1 <= n - 2 && (k + 1) % G == blk) {
            const double2* ck = col((k + 1) / G);
            double2* dst = a.ncol + (size_t)((k + 1) & 1) * n;
            for (int r = k + 1 + tid; r < n; r += kTriThreads) dst[r] = ck[r];
        }
        // P5
        dots(k);
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag)) return;
    }
    __syncthreads();
    if ((n - 1) % G == blk && tid == 0) a.d[n - 1] = col((n - 1) / G)[n - 1].x;
}

// Gram matrix of the conjugated projections: G_ij = sum_r b_i[r] conj(b_j[r]) (one block)
__global__ void gram_kernel(const double2* __restrict__ b, int64_t n, int np, double2* G) {
    __shared__ double s[kTriWarps][18];
    double acc[18];
    for (int q = 0; q < 18; ++q) acc[q] = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x)
        for (int i = 0; i < np; ++i)
            for (int j = 0; j < np; ++j) {
                const double2 bi = b[(size_t)i * n + r], bj = b[(size_t)j * n + r];
                acc[2 * (i * 3 + j)] += bi.x * bj.x + bi.y * bj.y;
                acc[2 * (i * 3 + j) + 1] += bi.y * bj.x - bi.x * bj.y;
            }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < 18; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) s[wid][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            x += s[w][2 * threadIdx.x];
            y += s[w][2 * threadIdx.x + 1];
        }
        G[threadIdx.x] = make_double2(x, y);
    }
}

// H0 = I - beta v v^H with H0 conj(b) = -phase ||b|| e_0 (one block)
__global__ void reflect0_kernel(const double2* __restrict__ b, int64_t n, double2* v, double* beta) {
    __shared__ double s[kTriWarps];
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc += b[r].x * b[r].x + b[r].y * b[r].y;
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    double nrm2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) nrm2 += s[w];
    const double nrm = sqrt(nrm2);
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double2 c = make_double2(b[r].x, -b[r].y);
        if (nrm2 == 0.0) {
            v[r] = make_double2(0.0, 0.0);
        } else if (r == 0) {
            const double ac = sqrt(c.x * c.x + c.y * c.y);
            const double2 ph = ac > 0.0 ? make_double2(c.x / ac, c.y / ac) : make_double2(1.0, 0.0);
            v[0] = make_double2(c.x + ph.x * nrm, c.y + ph.y * nrm);
        } else {
            v[r] = c;
        }
    }
    if (threadIdx.x == 0) {
        const double2 c0 = make_double2(b[0].x, -b[0].y);
        const double ac = sqrt(c0.x * c0.x + c0.y * c0.y);
        *beta = nrm2 == 0.0 ? 0.0 : 2.0 / (2.0 * nrm2 + 2.0 * nrm * ac);
    }
}

struct TriBounds {
    double gl, gu, tnorm, pivmin, tol;
    int m;           // T splits after row m-1 (first |e| <= tol), m = n when it does not
    float pivmin32;  // smallest pivot magnitude of the FP32 Sturm counts
};

// Gershgorin interval, deflation of negligible off-diagonals, e^2, and FP32
// copies of d and e^2 for the first rounds of the bisection (one block)
__global__ void tri_bounds_kernel(const double* __restrict__ d, const double* __restrict__ e, int64_t n, double* e2,
                                  float* d32, float* e2_32, TriBounds* out) {
    __shared__ double s_lo[kTriWarps], s_hi[kTriWarps], s_nm[kTriWarps], s_e[kTriWarps];
    __shared__ int s_m[kTriWarps];
    double lo = DBL_MAX, hi = -DBL_MAX, nm = 0.0, emax = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        nm = fmax(nm, fabs(d[i]) + r);
        if (i + 1 < n) emax = fmax(emax, e[i] * e[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        nm = fmax(nm, __shfl_xor_sync(0xffffffffu, nm, o));
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        s_lo[wid] = lo;
        s_hi[wid] = hi;
        s_nm[wid] = nm;
        s_e[wid] = emax;
    }
    __syncthreads();
    lo = DBL_MAX;
    hi = -DBL_MAX;
    nm = 0.0;
    emax = 0.0;
    for (int w = 0; w < nw; ++w) {
        lo = fmin(lo, s_lo[w]);
        hi = fmax(hi, s_hi[w]);
        nm = fmax(nm, s_nm[w]);
        emax = fmax(emax, s_e[w]);
    }
    const double tol = 64.0 * DBL_EPSILON * nm;
    int m = (int)n;
    for (int64_t i = threadIdx.x; i + 1 < n; i += blockDim.x) {
        const bool small = fabs(e[i]) <= tol;
        e2[i] = small ? 0.0 : e[i] * e[i];
        e2_32[i] = (float)e2[i];
        if (small && (int)i + 1 < m) m = (int)i + 1;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) d32[i] = (float)d[i];
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_m[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < nw; ++w) m = min(m, s_m[w]);
        TriBounds b;
        b.tnorm = nm;
        b.pivmin = DBL_MIN * fmax(1.0, emax);
        b.gl = lo - 2.0 * DBL_EPSILON * nm * (double)n - 2.0 * b.pivmin;
        b.gu = hi + 2.0 * DBL_EPSILON * nm * (double)n + 2.0 * b.pivmin;
        b.tol = tol;
        b.m = m;
        b.pivmin32 = FLT_MIN * (float)fmin(fmax(1.0, emax), 1e30);
        *out = b;
    }
}

// Number of eigenvalues below x of the tridiagonal rows [i0, i1): sign
// changes of the leading principal minors p_i = det(T[i0..i] - x), from the
// three-term recurrence p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (Sturm).
// No division (an FP64 divide costs about a thousand cycles of latency on
// this GPU); p_{i-1}, p_i are rescaled by an exact power of two every eight
// rows.  An exact zero p_i is replaced by -2^-200 p_{i-1}, as a zero pivot is
// replaced by a tiny negative one in the ratio form.
__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int i0, int i1,
                                           double x) {
    double pm = 1.0, p = __ldg(d + i0) - x;
    if ((__double_as_longlong(p) << 1) == 0) p = -0x1p-200;
    bool sp = neg_bit(p);
    int c = sp;
    for (int i = i0 + 1; i < i1; ++i) {
        double pn = fma(__ldg(d + i) - x, p, -__ldg(e2 + i - 1) * pm);
        if ((__double_as_longlong(pn) << 1) == 0) pn = -p * 0x1p-200;   // zero pivot -> -tiny (ratio p_i / p_{i-1})
        const bool sn = neg_bit(pn);
        c += sn != sp;
        sp = sn;
        pm = p;
        p = pn;
        if (((i - i0) & 7) == 0) {
            const int ex = (int)((__double_as_longlong(p) >> 52) & 0x7ff) - 1023;
            if (ex > 256 || ex < -256) {
                const double s = exp2i(-ex);
                p *= s;
                pm *= s;
            }
        }
    }
    return c;
}

// Number of eigenvalues below x of rows [i0, i1) in FP32, ratio form
// q_i = (d_i - x) - e_{i-1}^2 / q_{i-1} with pivots kept away from zero by
// pivmin (negative q counted).  The count is exact for a matrix within a few
// FP32 roundings of T (Kahan's backward analysis of the ratio recurrence), so
// a level bracketed by FP32 counts lies within 16 eps_32 (||T|| + |x|) of the
// bracket; the FP32 pipe is 64 times the FP64 one on this GPU.
__device__ __forceinline__ int sturm_count32(const float* __restrict__ d, const float* __restrict__ e2, int i0, int i1,
                                             float x, float pivmin) {
    float q = __ldg(d + i0) - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    int c = q < 0.f;
    for (int i = i0 + 1; i < i1; ++i) {
        q = (__ldg(d + i) - x) - __ldg(e2 + i - 1) / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.f;
    }
    return c;
}

// Sixteen lanes per level: 17-section of the Gershgorin interval with Sturm
// counts: 6 rounds in FP32 (from 2 ||T|| to about eps_32 ||T||), the bracket
// widened by the FP32 counts' backward error, then 9 rounds in FP64 to below
// eps ||T|| (17^9 > 1e11).  GB300 runs two FP64 lanes
// per clock per SM, so the cost is the chain of FP64 warp instructions each
// warp issues: fewer, wider rounds and one warp per SM sub-partition beat
// narrow bisection.  Every lane runs all rounds (uniform ballots).  Levels
// k < m belong to rows [0, m), the others to rows [m, n).
constexpr int kSect = 16;
__global__ void bisect_kernel(const double* __restrict__ d, const double* __restrict__ e2,
                              const float* __restrict__ d32, const float* __restrict__ e2_32, int64_t n,
                              const TriBounds* __restrict__ bnd, double* lam) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, sub = lane % kSect, base = lane - sub;
    const int64_t k = min(t / kSect, n - 1);
    const TriBounds b = *bnd;
    const int i0 = k < b.m ? 0 : b.m, i1 = k < b.m ? b.m : (int)n;
    const int kk = (int)(k - i0);
    float lof = (float)b.gl, hif = (float)b.gu;
    for (int it = 0; it < 6; ++it) {
        const float x = lof + (hif - lof) * (float)(sub + 1) * (1.0f / (kSect + 1));
        const int c = sturm_count32(d32, e2_32, i0, i1, x, b.pivmin32);
        const unsigned q = (__ballot_sync(0xffffffffu, c > kk) >> base) & ((1u << kSect) - 1u);
        const int ls = q ? __ffs(q) - 1 : kSect;   // first point above level kk
        const float xl = __shfl_sync(0xffffffffu, x, base + (ls > 0 ? ls - 1 : 0));
        const float xh = __shfl_sync(0xffffffffu, x, base + (ls < kSect ? ls : kSect - 1));
        if (ls > 0) lof = xl;
        if (ls < kSect) hif = xh;
    }
    const double del = 16.0 * FLT_EPSILON * (b.tnorm + fmax(fabs((double)lof), fabs((double)hif)));
    double lo = fmax(b.gl, (double)lof - del), hi = fmin(b.gu, (double)hif + del);
    for (int it = 0; it < 9; ++it) {
        const double x = lo + (hi - lo) * (double)(sub + 1) * (1.0 / (kSect + 1));
        const int c = sturm_count(d, e2, i0, i1, x);
        const unsigned q = (__ballot_sync(0xffffffffu, c > kk) >> base) & ((1u << kSect) - 1u);
        const int ls = q ? __ffs(q) - 1 : kSect;   // first point above level kk
        const double xl = __shfl_sync(0xffffffffu, x, base + (ls > 0 ? ls - 1 : 0));
        const double xh = __shfl_sync(0xffffffffu, x, base + (ls < kSect ? ls : kSect - 1));
        if (ls > 0) lo = xl;
        if (ls < kSect) hi = xh;
    }
    if (sub == 0 && t / kSect < n) lam[k] = 0.5 * (lo + hi);
}

// Squared first component of the eigenvector of rows [0, m) for level k < m,
// from the twisted factorisation T - lam = N_r Delta_r N_r^T at the twist
// index r with the smallest |gamma_r| (gamma_r = D+_r + D-_r - (d_r - lam));
// zero for levels of rows [m, n).  With z_r = 1, z_i = -L+_i z_{i+1} above r
// and z_{i+1} = -U-_i z_i below it, so
//   z_0^2 = prod_{i<r} L+_i^2,  sum_{i<r} z_i^2 = h_r,  sum_{i>r} z_i^2 = t_r
// with h_{i+1} = L+_i^2 (1 + h_i) and t_i = U-_i^2 (1 + t_{i+1}).
// A block of two warps takes 32 levels: warp 0 runs the top-down pass, warp
// 1 the bottom-up pass at the same time (each FP64 instruction of a warp
// costs the same whatever its active lanes, so the passes are split across
// warps, not lanes); both then scan half of the twist indices.
// st: scratch of 5 [m][n] arrays (level index fastest).
__global__ void __launch_bounds__(64) twisted_weights_kernel(const double* __restrict__ d, const double* __restrict__ e,
                                                             int64_t n, const TriBounds* __restrict__ bnd,
                                                             const double* __restrict__ lam, double* st, double* w) {
    __shared__ unsigned long long s_best[2][32];
    __shared__ int s_r[2][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * 32 + lane;
    const TriBounds b = *bnd;
    const int m = b.m;
    const bool act = k0 < m;
    const int64_t k = act ? k0 : 0;
    const double l = lam[k], piv = b.pivmin;
    double* Dp = st;
    double* Ph = st + (size_t)n * n;
    double* Hh = st + 2 * (size_t)n * n;
    double* Dm = st + 3 * (size_t)n * n;
    double* Tt = st + 4 * (size_t)n * n;
    if (act) {
        if (wid == 0) {   // top-down: D+_i, and P_i, h_i before row i
            double p = __ldg(d) - l, P = 1.0, h = 0.0;
            for (int i = 0; i + 1 < m; ++i) {
                if (fabs(p) < piv) p = -piv;
                Dp[(size_t)i * n + k] = p;
                Ph[(size_t)i * n + k] = P;
                Hh[(size_t)i * n + k] = h;
                const double L = __ldg(e + i) * rcp_nr(p);
                const double L2 = L * L;
                p = fma(-__ldg(e + i), L, __ldg(d + i + 1) - l);
                P *= L2;
                h = fma(L2, h, L2);
            }
            if (fabs(p) < piv) p = -piv;
            Dp[(size_t)(m - 1) * n + k] = p;
            Ph[(size_t)(m - 1) * n + k] = P;
            Hh[(size_t)(m - 1) * n + k] = h;
        } else {          // bottom-up: D-_i and t_i
            double q = __ldg(d + m - 1) - l, t = 0.0;
            Dm[(size_t)(m - 1) * n + k] = q;
            Tt[(size_t)(m - 1) * n + k] = 0.0;
            for (int i = m - 2; i >= 0; --i) {
                if (fabs(q) < piv) q = -piv;
                const double u = __ldg(e + i) * rcp_nr(q);
                q = fma(-u, __ldg(e + i), __ldg(d + i) - l);
                t = u * u * (1.0 + t);
                Dm[(size_t)i * n + k] = q;
                Tt[(size_t)i * n + k] = t;
            }
        }
    }
    __syncthreads();
    // twist index: smallest |gamma_i| over this warp's half (ties: lowest i)
    unsigned long long best = ~0ull;
    int rb = 0;
    if (act) {
        const int h0 = wid == 0 ? 0 : m / 2, h1 = wid == 0 ? m / 2 : m;
        for (int i = h0; i < h1; ++i) {
            const double g = Dp[(size_t)i * n + k] + Dm[(size_t)i * n + k] - (__ldg(d + i) - l);
            const unsigned long long ga = (unsigned long long)__double_as_longlong(g) & 0x7fffffffffffffffull;
            if (ga < best) {
                best = ga;
                rb = i;
            }
        }
    }
    s_best[wid][lane] = best;
    s_r[wid][lane] = rb;
    __syncthreads();
    if (wid == 0 && act) {
        const int r = s_best[1][lane] < s_best[0][lane] ? s_r[1][lane] : s_r[0][lane];
        const double P = Ph[(size_t)r * n + k], h = Hh[(size_t)r * n + k], t = Tt[(size_t)r * n + k];
        w[k] = P * rcp_nr(1.0 + h + t);
    } else if (wid == 0 && k0 < n) {
        w[k0] = 0.0;
    }
}

// ascending order of all levels (ties by index): a permutation even where the
// independently bisected levels of the two parts interleave; osc = scale * w
__global__ void rank_levels_kernel(const double* __restrict__ lam, const double* __restrict__ w, int64_t n,
                                   double scale, double* omega_out, double* osc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double x = lam[k];
    int64_t pos = 0;
    for (int64_t j = 0; j < n; ++j) {
        const double y = __ldg(lam + j);
        pos += (y < x) || (y == x && j < k);
    }
    omega_out[pos] = x;
    osc[pos] = scale * w[k];
}

__global__ void sum_kernel(const double* __restrict__ w, int64_t n, double* out) {
    __shared__ double s[kTriWarps];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += w[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s[i];
        *out = t;
    }
}

}  // namespace

size_t tridiag_scratch_bytes(int64_t n) {
    // v0 n, ncol 2n, xbuf 2n, spart 2 x 1024 (double2); d, e, e2, lam, w (n doubles); d32, e2_32 (n floats);
    // twisted passes 5 n*n doubles; 256-byte alignment of each piece
    return sizeof(double2) * (size_t)(5 * n + 2048) + sizeof(double) * (size_t)(5 * n + 5 * n * n) +
           sizeof(float) * (size_t)(2 * n) + 8192;
}

int tridiag_max_dim() { return 4736; }   // v, w and the next column of a step in 227 KB of shared memory

int launch_gram(const double2* b, int64_t n, int np, double2* G, cudaStream_t st) {
    if (np < 1 || np > 3) return fail(BSE_EINVAL, "gram of %d vectors", np);
    gram_kernel<<<1, kTriThreads, 0, st>>>(b, n, np, G);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

// Reduce the block h (n x n, ld n, device; overwritten in the global-memory
// variant) to T after the start reflector of b, then levels and weights.
int launch_tridiag_spectrum(double2* h, int64_t n, const double2* b, double scale, void* scratch, double* omega_out,
                            double* osc, double* wsum, int* err, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1) {
    if (n < 1 || n > tridiag_max_dim()) return fail(BSE_EUNSUPPORTED, "tridiagonal path: n = %lld", (long long)n);
    char* p = (char*)scratch;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)q;
    };
    double2* v0 = (double2*)take(sizeof(double2) * n);
    double2* ncol = (double2*)take(sizeof(double2) * 2 * n);
    double2* xbuf = (double2*)take(sizeof(double2) * 2 * n);
    double2* spart = (double2*)take(sizeof(double2) * 2048);
    double* d = (double*)take(sizeof(double) * n);
    double* e = (double*)take(sizeof(double) * n);
    double* e2 = (double*)take(sizeof(double) * n);
    float* d32 = (float*)take(sizeof(float) * n);
    float* e2_32 = (float*)take(sizeof(float) * n);
    double* lam = (double*)take(sizeof(double) * n);
    double* w = (double*)take(sizeof(double) * n);
    double* beta0 = (double*)take(sizeof(double));
    TriBounds* bnd = (TriBounds*)take(sizeof(TriBounds));
    unsigned* bar = (unsigned*)take(sizeof(unsigned));
    double* dp = (double*)take(sizeof(double) * 5 * n * n);

    int dev = 0, sms = 0, maxsm = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BSE_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int G = (int)std::min<int64_t>(sms, std::max<int64_t>(1, (n + 3) / 4));
    const size_t static_smem = sizeof(double2) * (kTriWarps + 3) + sizeof(double) * kTriWarps + 64;
    const size_t vec_bytes = sizeof(double2) * 3 * (size_t)n;   // v, w and the next column of a step
    const size_t cols_bytes = sizeof(double2) * (size_t)((n - 1) / G + 1) * n;
    const bool smem = vec_bytes + cols_bytes + static_smem <= (size_t)maxsm;
    if (!smem) G = sms;
    if (vec_bytes + static_smem > (size_t)maxsm)
        return fail(BSE_EUNSUPPORTED, "tridiagonal path: n = %lld exceeds shared memory", (long long)n);

    BSE_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    BSE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    BSE_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, st));
    reflect0_kernel<<<1, kTriThreads, 0, st>>>(b, n, v0, beta0);
    note_launch();
    BSE_CUDA(cudaGetLastError());

    TriArgs a;
    a.A = h;
    a.n = n;
    a.v0 = v0;
    a.beta0 = beta0;
    a.ncol = ncol;
    a.xbuf = xbuf;
    a.spart = spart;
    a.d = d;
    a.e = e;
    a.bar = bar;
    a.err = err;
    void* args[] = {&a};
    const size_t dyn = vec_bytes + (smem ? cols_bytes : 0);
    const void* fn = smem ? (const void*)tridiag_kernel<true> : (const void*)tridiag_kernel<false>;
    BSE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTriThreads, dyn));
    if (per_sm < 1 || G > per_sm * sms) return fail(BSE_EUNSUPPORTED, "tridiagonal kernel cannot be co-resident");
    if (ev0) BSE_CUDA(cudaEventRecord(ev0, st));
    BSE_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kTriThreads), args, dyn, st));
    note_launch();
    if (ev1) BSE_CUDA(cudaEventRecord(ev1, st));

    tri_bounds_kernel<<<1, kTriThreads, 0, st>>>(d, e, n, e2, d32, e2_32, bnd);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    bisect_kernel<<<(unsigned)((kSect * n + 31) / 32), 32, 0, st>>>(d, e2, d32, e2_32, n, bnd, lam);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    twisted_weights_kernel<<<(unsigned)((n + 31) / 32), 64, 0, st>>>(d, e, n, bnd, lam, dp, w);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    rank_levels_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(lam, w, n, scale, omega_out, osc);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    sum_kernel<<<1, kTriThreads, 0, st>>>(w, n, wsum);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

}  // namespace bse
