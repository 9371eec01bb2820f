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
// scalar, and one grid barrier per step orders the reflector and x = tau A v.
// The reduction computes in double-float arithmetic (dfloat.h) on the FP32
// pipe, 64 times wider than GB300's FP64 pipe; the block is read in FP64 and
// T is written in FP64.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "dfloat.h"
#include "fp64_fast.h"
#include "grid_sync.h"
#include "internal.h"
#include "reflector.h"

namespace bse {

namespace {

constexpr int kTriThreads = 256;
constexpr int64_t kTwoStageFrom = 1800;   // the automatic choice takes the two-stage reduction from this size
constexpr int kTriWarps = kTriThreads / 32;
constexpr int kChunk = 8;                 // columns updated together

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rank-2 update A_rc -= v_r conj(w_c) + w_r conj(v_c) of a chunk of columns,
// rows r0 + t, r0 + t + nt, ...
// kTwo (columns in global memory): two rows per iteration, all their loads
// issued before the arithmetic, so that more bytes are in flight per thread
template <int NC, bool kTwo>
__device__ __forceinline__ void chunk_update(cdf* cb, size_t cs, const cdf* V, const cdf* W, const int* jcol,
                                             int r0, int n, int t, int nt) {
    cdf vj[NC], wj[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        vj[c] = V[jcol[c]];
        wj[c] = W[jcol[c]];
    }
    int r = r0 + t;
    if (kTwo)
        for (; r + nt < n; r += 2 * nt) {
            cdf q0[NC], q1[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                q0[c] = cb[c * cs + r];
                q1[c] = cb[c * cs + r + nt];
            }
            const cdf v0 = V[r], w0 = W[r], v1 = V[r + nt], w1 = W[r + nt];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                cb[c * cs + r] = cdf_rank2(q0[c], v0, w0, wj[c], vj[c]);
                cb[c * cs + r + nt] = cdf_rank2(q1[c], v1, w1, wj[c], vj[c]);
            }
        }
    for (; r < n; r += nt) {
        const cdf v = V[r], w = W[r];
#pragma unroll
        for (int c = 0; c < NC; ++c) cb[c * cs + r] = cdf_rank2(cb[c * cs + r], v, w, wj[c], vj[c]);
    }
}

#define BSE_NC_DISPATCH(nc, two, F, ...)          \
    switch (nc) {                                  \
        case 1: F<1, two>(__VA_ARGS__); break;     \
        case 2: F<2, two>(__VA_ARGS__); break;     \
        case 3: F<3, two>(__VA_ARGS__); break;     \
        case 4: F<4, two>(__VA_ARGS__); break;     \
        case 5: F<5, two>(__VA_ARGS__); break;     \
        case 6: F<6, two>(__VA_ARGS__); break;     \
        case 7: F<7, two>(__VA_ARGS__); break;     \
        default: F<8, two>(__VA_ARGS__); break;    \
    }

struct TriArgs {
    double2* A;           // n x n column-major, leading dimension n; the global variant rewrites it in place in
                          // double-float (same 16 bytes per element) and updates it there
    int64_t n;
    const double2* v0;    // initial reflector
    const double* beta0;  // its (real) scalar
    cdf* ncol;            // [2][n] the next column to be reflected, published by its owner, by parity
    cdf* xbuf;            // [2][n] x = tau A v, by step parity
    cdf* spart;           // [2][G] per-CTA parts of x^H v, by step parity
    double* d;            // [n] diagonal of T
    double* e;            // [n] off-diagonal of T (e[n-1] unused)
    unsigned* bar;        // barrier counter, zero on entry
    int* err;             // error flag, zero on entry
    long spin;            // polls of a grid barrier before it gives up
};


// One grid barrier per reflection step s (H(s) = I - tau v v^H on rows >= s+1,
// s = -1 being the start reflector H0 on all rows), k = s+1:
//   P1  x(s), the parts of x^H v from all CTAs and the published column k:
//       alpha = -tau (x^H v)/2
//   P2  w = x + alpha v; column k updated by this step,
//       c_r - v_r conj(w_k) - w_r conj(v_k), and its squared norm below row k+1
//   P3  warp 0: reflector k from it (zlarfg convention, v_{k+1} = 1);
//       warps 1-7 at the same time: own columns j >= k,
//       A_rj -= v_r conj(w_j) + w_r conj(v_j), rows r >= k
//   P4  the new reflector v(k) in place of column k; the owner of column k+1
//       publishes it (its state before step k)
//   P5  x(k)_j = tau(k) sum_r conj(A_rj) v(k)_r for own columns j > k (Hermitian:
//       (A v)_j is a column dot product) and this CTA's part of x^H v
//   grid barrier
template <bool kSmem>
__global__ void __launch_bounds__(kTriThreads, 1) tridiag_kernel(TriArgs a) {
    extern __shared__ __align__(16) cdf s_dyn[];
    __shared__ cdf s_part[kTriWarps];
    __shared__ cdf s_alpha, s_tau, s_inv;
    __shared__ int s_flag;

    const int n = (int)a.n;
    const int G = gridDim.x, blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ncl = blk < n ? (n - 1 - blk) / G + 1 : 0;
    cdf* V = s_dyn;                       // reflector of the step
    cdf* W = s_dyn + n;                   // w of the step
    cdf* C = s_dyn + 2 * (size_t)n;       // next column, then its update, then the next reflector
    cdf* s_cols = s_dyn + 3 * (size_t)n;
    cdf* gA = reinterpret_cast<cdf*>(a.A);
    auto col = [&](int l) -> cdf* {
        return kSmem ? s_cols + (size_t)l * n : gA + (size_t)(blk + l * G) * n;
    };
    const size_t cstride = kSmem ? (size_t)n : (size_t)G * n;
    // own columns in double-float; in the global variant each element is read
    // and rewritten in place by the same thread
    for (int l = 0; l < ncl; ++l) {
        const double2* src = a.A + (size_t)(blk + l * G) * n;
        cdf* dst = col(l);
        for (int r = tid; r < n; r += kTriThreads) {
            const double2 z = src[r];
            dst[r] = cdf_from(z);
        }
    }
    for (int r = tid; r < n; r += kTriThreads) V[r] = cdf_from(__ldcg(a.v0 + r));
    if (tid == 0) s_tau = cdf_from(make_double2(__ldcg(a.beta0), 0.0));
    __syncthreads();
    // column 0 as it is before the start reflector
    if (blk == 0)
        for (int r = tid; r < n; r += kTriThreads) a.ncol[r] = col(0)[r];
    unsigned nbar = 0;

    // P5 for reflector k (rows > k; k = -1: all rows) with reflector vector Vk:
    // one warp per column
    auto dots = [&](int k, const cdf* Vk) {
        const int r0 = k + 1;
        const cdf tau = s_tau;
        const int l0 = blk >= r0 ? 0 : (r0 - blk + G - 1) / G;
        cdf* xb = a.xbuf + (size_t)(k & 1) * n;
        cdf sw = cdf_zero();
        for (int l = l0 + wid; l < ncl; l += kTriWarps) {
            const cdf* cl = col(l);
            cdf acc = cdf_zero(), acc2 = cdf_zero();
            int r = r0 + lane;
            if (!kSmem)   // columns in global memory: four rows' loads in flight per lane
                for (; r + 96 < n; r += 128) {
                    const cdf a0 = cl[r], a1 = cl[r + 32], a2 = cl[r + 64], a3 = cl[r + 96];
                    acc = cdf_dot_acc(acc, a0, Vk[r]);
                    acc2 = cdf_dot_acc(acc2, a1, Vk[r + 32]);
                    acc = cdf_dot_acc(acc, a2, Vk[r + 64]);
                    acc2 = cdf_dot_acc(acc2, a3, Vk[r + 96]);
                }
            for (; r + 32 < n; r += 64) {
                acc = cdf_dot_acc(acc, cl[r], Vk[r]);
                acc2 = cdf_dot_acc(acc2, cl[r + 32], Vk[r + 32]);
            }
            if (r < n) acc = cdf_dot_acc(acc, cl[r], Vk[r]);
            acc = cdf_warp_sum(cdf_add(acc, acc2));
            if (lane == 0) {
                const int j = blk + l * G;
                const cdf x = cdf_mul(tau, acc);
                xb[j] = x;
                sw = cdf_dot_acc(sw, x, Vk[j]);
            }
        }
        if (lane == 0) s_part[wid] = sw;
        __syncthreads();
        if (tid == 0) {
            cdf sp = s_part[0];
            for (int w = 1; w < kTriWarps; ++w) sp = cdf_add(sp, s_part[w]);
            a.spart[(size_t)(k & 1) * G + blk] = sp;
        }
    };

    dots(-1, V);
    if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;

    for (int s = -1; s <= n - 2; ++s) {
        const int k = s + 1;   // first row of this step's reflector, column reflected next
        const bool more = s < n - 2;
        // P1
        const cdf* xb = a.xbuf + (size_t)(s & 1) * n;
        const cdf* nc_src = a.ncol + (size_t)(k & 1) * n;
        const cdf xk = __ldcg(xb + k);
        for (int r = k + tid; r < n; r += kTriThreads) {
            W[r] = __ldcg(xb + r);
            if (more) C[r] = __ldcg(nc_src + r);
        }
        if (wid == 0) {
            const cdf* sp = a.spart + (size_t)(s & 1) * G;
            cdf acc = cdf_zero();
            for (int b = lane; b < G; b += 32) acc = cdf_add(acc, __ldcg(sp + b));
            acc = cdf_warp_sum(acc);
            if (lane == 0) {
                const cdf al = cdf_mul(s_tau, acc);
                s_alpha = make_float4(-0.5f * al.x, -0.5f * al.y, -0.5f * al.z, -0.5f * al.w);
            }
        }
        __syncthreads();
        // P2
        const cdf alpha = s_alpha;
        const cdf vk = V[k];
        const cdf wk = cdf_fma(xk, alpha, vk);
        float sg = 0.f, sgl = 0.f;
        for (int r = k + tid; r < n; r += kTriThreads) {
            const cdf v = V[r];
            const cdf w = cdf_fma(W[r], alpha, v);
            W[r] = w;
            if (more) {
                const cdf cr = cdf_rank2(C[r], v, w, wk, vk);
                C[r] = cr;
                if (r >= k + 2) {
                    df_acc(sg, sgl, cr.x, cr.y, cr.x, cr.y);
                    df_acc(sg, sgl, cr.z, cr.w, cr.z, cr.w);
                }
            }
        }
        if (more) {
            const float2 f = df_fin(sg, sgl);
            const cdf t = cdf_warp_sum(make_float4(f.x, f.y, 0.f, 0.f));
            if (lane == 0) s_part[wid] = t;
        }
        __syncthreads();
        // P3
        if (wid == 0) {
            if (more && lane == 0) {
                float2 sigma = make_float2(s_part[0].x, s_part[0].y);
                for (int w = 1; w < kTriWarps; ++w) sigma = df_add(sigma, make_float2(s_part[w].x, s_part[w].y));
                cdf tau, inv;
                float2 beta;
                reflector(C[k + 1], sigma, tau, inv, beta);
                s_tau = tau;
                s_inv = inv;
                if (blk == 0) {
                    a.d[k] = df_to(make_float2(C[k].x, C[k].y));
                    a.e[k] = df_to(beta);
                }
            }
        } else {
            const int l0 = blk >= k ? 0 : (k - blk + G - 1) / G;
            for (int c0 = l0; c0 < ncl; c0 += kChunk) {
                const int nc = min(kChunk, ncl - c0);
                int jcol[kChunk];
#pragma unroll
                for (int c = 0; c < kChunk; ++c) jcol[c] = blk + (c0 + c) * G;
                BSE_NC_DISPATCH(nc, !kSmem, chunk_update, col(c0), cstride, V, W, jcol, k, n, tid - 32,
                                kTriThreads - 32)
            }
        }
        if (!more) break;
        __syncthreads();
        // P4
        {
            const cdf inv = s_inv;
            for (int r = k + 1 + tid; r < n; r += kTriThreads)
                C[r] = r == k + 1 ? make_float4(1.f, 0.f, 0.f, 0.f) : cdf_mul(C[r], inv);
        }
        if (k + 1 <= n - 2 && (k + 1) % G == blk) {
            const cdf* ck = col((k + 1) / G);
            cdf* dst = a.ncol + (size_t)((k + 1) & 1) * n;
            for (int r = k + 1 + tid; r < n; r += kTriThreads) dst[r] = ck[r];
        }
        __syncthreads();
        // P5
        dots(k, C);
        cdf* t = V;
        V = C;
        C = t;
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;
    }
    __syncthreads();
    if ((n - 1) % G == blk && tid == 0) {
        const cdf z = col((n - 1) / G)[n - 1];
        a.d[n - 1] = df_to(make_float2(z.x, z.y));
    }
}

// ---------------------------------------------------------------------------
// Blocked reduction for blocks whose columns live in global memory.
//
// The same reflectors as tridiag_kernel, applied in panels of kNb: within a
// panel the trailing matrix A is left as it was at the panel's start, and the
// reflectors' two-sided updates A_cur = A - sum_l (v_l w_l^H + w_l v_l^H) are
// carried as corrections.  Step s (reflector s acts on rows > s; s = -1 is the
// start reflector on all rows), with l reflectors of the panel before it:
//   phase 1  reflector s from the current column s (published in phase 2 of
//            step s - 1); z_i = sum_r conj(A[r,i]) v_r for own columns i > s
//            (A Hermitian: (A v)_i is a column dot product), started on the
//            unscaled column while one warp forms the reflector's scalars;
//            s1_b = W_b^H v, s2_b = V_b^H v by CTAs b < 2 l
//   grid barrier
//   phase 2  y = tau (z - V s1 - W s2), alpha = -tau/2 y^H v with
//            y^H v = conj(tau) (z^H v - 2 Re s1^H s2); w = y + alpha v for own
//            indices, stored as column l of W (v as column l of V); the
//            current column k = s + 1 on own rows, A[:,k] - sum_{l' <= l}
//            (V_l' conj(W[k,l']) + W_l' conj(V[k,l'])), published with its
//            squared norm below row k + 1
//   grid barrier
//   panel end: A -= V W^H + W V^H on own columns and the trailing rows
//            (rank 2 kNb, register-blocked, double-float on the FP32 pipe)
// Per step the trailing matrix is read once (the dot products) instead of
// being read, written and read again by a rank-2 update and the dot products.
// ---------------------------------------------------------------------------
constexpr int kNb = 32;           // reflectors per panel
constexpr int kHerCols = 12;      // own columns updated together in the panel-end update

struct TriBArgs {
    cdf* A;               // n x n column-major; the FP64 block on entry, rewritten in place in double-float
    int64_t n;
    const double2* v0;    // start reflector (all rows) and its scalar
    const double* beta0;
    cdf* V;               // [kNb][n] the panel's reflectors: row i of reflector l at l * n + i
    cdf* W;               // [kNb][n] their w vectors
    cdf* ncol;            // [n] the current column of the next reflector (rows >= its index)
    float2* npart;        // [G] per-CTA parts of its squared norm below the subdiagonal
    cdf* zbuf;            // [2][n] the unscaled dot zr_i and the row s+1 term t_i of z_i = t_i + inv zr_i
    cdf* zpart;           // [G][4] per-CTA sums for z^H v: sum conj(t_i) c_i, sum conj(zr_i) c_i over own
                          // i >= s+2 (c the current column), and conj(t_i), conj(zr_i) of i = s+1
    cdf* sdot;            // [2][2 kNb] s1 (first kNb entries) and s2: unscaled sums and row s+1 terms
    double* d;            // [n] diagonal of T
    double* e;            // [n] off-diagonal of T
    unsigned* bar;        // barrier counter, zero on entry
    int* err;             // error flag, zero on entry
    long spin;            // polls of a grid barrier before it gives up
    int s_begin, s_end;   // the steps of this launch: s_begin <= s < s_end (s = -1: the start reflector)
    int tc_update;        // 1: the panel-end update is left to the tensor-core kernels between launches
    int resident_from;    // columns i >= resident_from are read with normal L2 priority (they stay in
                          // L2 from step to step), the others streamed with evict-first loads
    int stage_rows;       // rows per shared-memory stage of the column dot products (0: loads to registers)
};

// dynamic shared memory of the blocked kernel (cdf units): the staged column
// (n); per own column m the panel's W[i,l] and V[i,l] (2 kNb), its z, the row
// s+1 term of its dot, its v and w, and its entry of the next current column
// (5); s1, s2 and the current column's coefficients (4 (kNb + 1))
__host__ __device__ inline size_t tri_blocked_smem(int64_t n, int G) {
    const int64_t ncl = (n + G - 1) / G;
    return sizeof(cdf) * (size_t)(n + ncl * (2 * kNb + 5) + 4 * (kNb + 1)) + 64;
}

__device__ __forceinline__ cdf cdf_conj(cdf a) { return make_float4(a.x, a.y, -a.z, -a.w); }
__device__ __forceinline__ cdf cdf_neg(cdf a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

// a load of the streamed trailing matrix: marked evict-first in L2, so that the
// hundreds of MB read per step do not push the kernel's instructions and the
// panel's small vectors out of L2 (a refetch from saturated HBM costs tens of
// microseconds on the step's critical path)
template <bool kStream>
__device__ __forceinline__ cdf ld_col(const cdf* p) { return kStream ? __ldcs(p) : __ldcg(p); }

// sum_{r >= r0} conj(x[r]) c[r] over a column x in global memory, lanes over
// rows, sixteen rows' loads in flight per lane; reduced over the warp (used when
// shared memory has no room for the staged form below)
template <bool kStream>
__device__ __forceinline__ cdf warp_coldot(const cdf* __restrict__ x, const cdf* c, int r0, int n, int lane) {
    cdf acc0 = cdf_zero(), acc1 = cdf_zero(), acc2 = cdf_zero(), acc3 = cdf_zero();
    int r = r0 + lane;
    // sixteen rows' loads in flight per lane (8 KB per warp) while the column streams from HBM
    for (; r + 480 < n; r += 512) {
        cdf q[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) q[u] = ld_col<kStream>(x + r + 32 * u);
#pragma unroll
        for (int u = 0; u < 16; u += 4) {
            acc0 = cdf_dot_acc(acc0, q[u], c[r + 32 * u]);
            acc1 = cdf_dot_acc(acc1, q[u + 1], c[r + 32 * u + 32]);
            acc2 = cdf_dot_acc(acc2, q[u + 2], c[r + 32 * u + 64]);
            acc3 = cdf_dot_acc(acc3, q[u + 3], c[r + 32 * u + 96]);
        }
    }
    for (; r + 96 < n; r += 128) {
        const cdf q0 = ld_col<kStream>(x + r), q1 = ld_col<kStream>(x + r + 32), q2 = ld_col<kStream>(x + r + 64),
                  q3 = ld_col<kStream>(x + r + 96);
        acc0 = cdf_dot_acc(acc0, q0, c[r]);
        acc1 = cdf_dot_acc(acc1, q1, c[r + 32]);
        acc2 = cdf_dot_acc(acc2, q2, c[r + 64]);
        acc3 = cdf_dot_acc(acc3, q3, c[r + 96]);
    }
    for (; r < n; r += 32) acc0 = cdf_dot_acc(acc0, ld_col<kStream>(x + r), c[r]);
    return cdf_warp_sum(cdf_add(cdf_add(acc0, acc1), cdf_add(acc2, acc3)));
}

// 16-byte asynchronous copies global -> shared (L2 only), optionally with an evict-first L2 policy
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16_ef(void* dst, const void* src, uint64_t pol) {
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// The same dot product with the column streamed through three shared-memory
// stages of R rows per warp (R a multiple of 32): while a stage is multiplied
// the next two are in flight, without holding registers, so that the warp's
// HBM or L2 latency overlaps its double-float arithmetic.  Each lane copies and
// reads only its own rows (r = base + lane + 32 u), so no warp synchronisation
// is needed; every stage commits a copy group, empty or not.
__device__ __forceinline__ cdf warp_coldot_staged(const cdf* __restrict__ x, const cdf* c, int r0, int n, int lane,
                                               cdf* stg, int R, bool stream, uint64_t pol) {
    cdf acc0 = cdf_zero(), acc1 = cdf_zero(), acc2 = cdf_zero(), acc3 = cdf_zero();
    const int nst = (n - r0 + R - 1) / R;
    auto issue = [&](int st) {
        if (st < nst) {
            cdf* b = stg + (st % 3) * R;
            const int base = r0 + st * R;
            const int lim = min(R, n - base);
            if (stream)
                for (int u = lane; u < lim; u += 32) cp_async16_ef(b + u, x + base + u, pol);
            else
                for (int u = lane; u < lim; u += 32) cp_async16(b + u, x + base + u);
        }
        cp_async_commit();
    };
    issue(0);
    issue(1);
    for (int st = 0; st < nst; ++st) {
        issue(st + 2);
        cp_async_wait<2>();   // this lane's copies of stage st have landed
        const cdf* b = stg + (st % 3) * R;
        const int base = r0 + st * R;
        const int lim = min(R, n - base);
        int u = lane;
        for (; u + 96 < lim; u += 128) {
            acc0 = cdf_dot_acc(acc0, b[u], c[base + u]);
            acc1 = cdf_dot_acc(acc1, b[u + 32], c[base + u + 32]);
            acc2 = cdf_dot_acc(acc2, b[u + 64], c[base + u + 64]);
            acc3 = cdf_dot_acc(acc3, b[u + 96], c[base + u + 96]);
        }
        for (; u < lim; u += 32) acc0 = cdf_dot_acc(acc0, b[u], c[base + u]);
    }
    cp_async_wait<0>();
    return cdf_warp_sum(cdf_add(cdf_add(acc0, acc1), cdf_add(acc2, acc3)));
}

__global__ void __launch_bounds__(kTriThreads, 1) tridiag_blocked_kernel(TriBArgs a) {
    extern __shared__ __align__(16) cdf s_dyn[];
    __shared__ cdf s_tau, s_inv, s_alpha;
    __shared__ cdf s_zk;                     // z_k of the current column's index
    __shared__ cdf s_zp[kTriWarps][4];       // per-warp parts of the z^H v sums
    __shared__ float2 s_nrm[kTriWarps];
    __shared__ int s_next, s_flag;

    const int n = (int)a.n;
    const int G = gridDim.x, blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ncl = blk < n ? (n - 1 - blk) / G + 1 : 0;
    cdf* Cs = s_dyn;                                   // [n] the staged column (or v0)
    cdf* WV = Cs + n;                                  // [ncl][2 kNb]: W[i,l] then V[i,l] of own index i
    cdf* zown = WV + (size_t)ncl * 2 * kNb;            // [ncl] z_i (unscaled sum, then z)
    cdf* ztop = zown + ncl;                            // [ncl] conj(A[s+1, i])
    cdf* vown = ztop + ncl;                            // [ncl]
    cdf* wown = vown + ncl;                            // [ncl]
    cdf* colk = wown + ncl;                            // [ncl] A[i, k] of the next current column, own rows
    cdf* s12 = colk + ncl;                             // [2 (kNb + 1)]: s1 then s2
    cdf* cwv = s12 + 2 * (kNb + 1);                    // [2 (kNb + 1)]: W[k,l'] then V[k,l']
    cdf* stg = s_dyn + tri_blocked_smem(n, G) / sizeof(cdf) + (size_t)wid * 3 * a.stage_rows;   // this warp's stages
    const uint64_t pol = evict_first_policy();
    cdf* gA = a.A;
    auto col = [&](int i) -> cdf* { return gA + (size_t)i * n; };
    auto WVo = [&](int m, int l2) -> cdf& { return WV[(size_t)m * 2 * kNb + l2]; };

    // own columns in double-float, in place (same 16 bytes per element), at the first launch
    if (a.s_begin < 0)
        for (int m = 0; m < ncl; ++m) {
            const double2* src = reinterpret_cast<const double2*>(col(blk + m * G));
            cdf* dst = col(blk + m * G);
            for (int r = tid; r < n; r += kTriThreads) {
                const double2 z = src[r];
                dst[r] = cdf_from(z);
            }
        }
    unsigned nbar = 0;

    for (int s = a.s_begin; s < a.s_end; ++s) {
        const int k = s + 1;
        const int l = (s + 1) % kNb;     // reflectors of the panel before this one
        const int m0 = blk > s ? 0 : (s - blk) / G + 1;   // own indices i > s (= own rows i >= k)
        const int nown = ncl - m0;
        // ---------------- phase 1 ----------------
        // stage the current column (rows >= s) or the start reflector
        if (s < 0) {
            for (int r = tid; r < n; r += kTriThreads) Cs[r] = cdf_from(__ldcg(a.v0 + r));
        } else {
            for (int r = s + tid; r < n; r += kTriThreads) Cs[r] = __ldcg(a.ncol + r);
        }
        if (tid == 0) s_next = 0;
        __syncthreads();
        // own columns i > s, then the dots s_q, q = blk, blk + G, ... < 2 l
        const int nsq = blk < 2 * l ? (2 * l - 1 - blk) / G + 1 : 0;
        const int ntask = nown + nsq;
        const int r0 = s < 0 ? 0 : s + 2;
        if (wid == 0 && s >= 0) {   // the reflector's scalars (zlarfg convention, v_{s+1} = 1)
            float2 sg = make_float2(0.f, 0.f);
            for (int b = lane; b < G; b += 32) sg = df_add(sg, __ldcg(a.npart + b));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                sg = df_add(sg, make_float2(__shfl_xor_sync(0xffffffffu, sg.x, o), __shfl_xor_sync(0xffffffffu, sg.y, o)));
            if (lane == 0) {
                cdf tau, inv;
                float2 beta;
                reflector(Cs[s + 1], sg, tau, inv, beta);
                s_tau = tau;
                s_inv = inv;
                if (blk == 0) {
                    a.d[s] = df_to(make_float2(Cs[s].x, Cs[s].y));
                    a.e[s] = df_to(beta);
                }
            }
            __syncwarp();
        } else if (tid == 0 && s < 0) {
            s_tau = cdf_from(make_double2(__ldcg(a.beta0), 0.0));
            s_inv = make_float4(1.f, 0.f, 0.f, 0.f);
        }
        // dot tasks, taken dynamically (warp 0 joins once the reflector is done).  A column task
        // publishes the unscaled sum zr_i and the row s+1 term t_i = conj(A[s+1,i]) (z_i = t_i +
        // inv zr_i once the reflector is known), fetches the entry A[i,k] of the next current
        // column and adds to this warp's parts of z^H v = sum_i conj(z_i) v_i, which with
        // v_i = inv c_i (i >= s+2), v_{s+1} = 1 is inv sum conj(t_i) c_i + |inv|^2 sum conj(zr_i) c_i
        // + conj(t_{s+1}) + conj(inv) conj(zr_{s+1}).  An s task publishes the same pair for s_q.
        cdf p0 = cdf_zero(), p1 = cdf_zero(), p2 = cdf_zero(), p3 = cdf_zero();
        for (;;) {
            int t = 0;
            if (lane == 0) t = atomicAdd(&s_next, 1);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= ntask) break;
            if (t < nown) {
                const int m = m0 + t;
                const int i = blk + m * G;
                const cdf* x = col(i);
                cdf top = cdf_zero(), ck = cdf_zero();
                if (lane == 0) {
                    if (s >= 0) top = cdf_conj(__ldcg(x + s + 1));
                    if (l > 0) ck = __ldcg(col(k) + i);   // column k is not written during a panel
                }
                const bool stream = i < a.resident_from;
                const cdf zr = a.stage_rows > 0 ? warp_coldot_staged(x, Cs, r0, n, lane, stg, a.stage_rows, stream, pol)
                               : stream         ? warp_coldot<true>(x, Cs, r0, n, lane)
                                                : warp_coldot<false>(x, Cs, r0, n, lane);
                if (lane == 0) {
                    zown[m] = zr;
                    ztop[m] = top;
                    colk[m] = ck;
                    a.zbuf[i] = zr;
                    a.zbuf[n + i] = top;
                    if (s < 0) {                       // start reflector: v = v0, z = zr
                        p1 = cdf_dot_acc(p1, zr, Cs[i]);
                    } else if (i >= s + 2) {
                        p0 = cdf_dot_acc(p0, top, Cs[i]);
                        p1 = cdf_dot_acc(p1, zr, Cs[i]);
                    } else {                           // i = s + 1: conj(z) = conj(t) + conj(inv) conj(zr)
                        p2 = cdf_conj(top);
                        p3 = cdf_conj(zr);
                    }
                }
            } else {
                const int q = blk + (t - nown) * G;   // s1_q (q < l) or s2_{q - l}
                const cdf* x = q < l ? a.W + (size_t)q * n : a.V + (size_t)(q - l) * n;
                cdf top = cdf_zero();
                if (lane == 0 && s >= 0) top = cdf_conj(__ldcg(x + s + 1));
                const cdf sr = warp_coldot<false>(x, Cs, r0, n, lane);
                if (lane == 0) {
                    const int o = q < l ? q : kNb + q - l;
                    a.sdot[o] = sr;
                    a.sdot[2 * kNb + o] = top;
                }
            }
        }
        if (lane == 0) {
            s_zp[wid][0] = p0;
            s_zp[wid][1] = p1;
            s_zp[wid][2] = p2;
            s_zp[wid][3] = p3;
        }
        __syncthreads();
        if (wid == 0 && lane < 4) {
            cdf sum = s_zp[0][lane];
            for (int w = 1; w < kTriWarps; ++w) sum = cdf_add(sum, s_zp[w][lane]);
            a.zpart[(size_t)blk * 4 + lane] = sum;
        }
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;

        // ---------------- phase 2 ----------------
        const cdf tau = s_tau, inv = s_inv;
        if (wid == 0) {   // z^H v, s1, s2, Re s1^H s2 and alpha
            cdf q0 = cdf_zero(), q1 = cdf_zero(), q2 = cdf_zero(), q3 = cdf_zero();
            for (int b = lane; b < G; b += 32) {
                const cdf* zp = a.zpart + (size_t)b * 4;
                q0 = cdf_add(q0, __ldcg(zp));
                q1 = cdf_add(q1, __ldcg(zp + 1));
                q2 = cdf_add(q2, __ldcg(zp + 2));
                q3 = cdf_add(q3, __ldcg(zp + 3));
            }
            cdf s1 = cdf_zero(), s2 = cdf_zero();
            if (lane < l) {
                const cdf r1 = __ldcg(a.sdot + lane), t1 = __ldcg(a.sdot + 2 * kNb + lane);
                const cdf r2 = __ldcg(a.sdot + kNb + lane), t2 = __ldcg(a.sdot + 3 * kNb + lane);
                s1 = s >= 0 ? cdf_fma(t1, inv, r1) : r1;
                s2 = s >= 0 ? cdf_fma(t2, inv, r2) : r2;
                s12[lane] = s1;
                s12[kNb + 1 + lane] = s2;
            }
            q0 = cdf_warp_sum(q0);
            q1 = cdf_warp_sum(q1);
            q2 = cdf_warp_sum(q2);
            q3 = cdf_warp_sum(q3);
            const cdf cr = cdf_warp_sum(cdf_dot_acc(cdf_zero(), s1, s2));   // s1^H s2
            if (lane == 0) {
                // z^H v = inv q0 + |inv|^2 q1 + q2 + conj(inv) q3 (start reflector: q1)
                cdf zv;
                if (s >= 0) {
                    const cdf ii = cdf_dot_acc(cdf_zero(), inv, inv);   // |inv|^2
                    zv = cdf_fma(cdf_fma(cdf_fma(q2, inv, q0), ii, q1), cdf_conj(inv), q3);
                } else {
                    zv = q1;
                }
                // y^H v = conj(tau) (z^H v - 2 Re s1^H s2); alpha = -tau/2 y^H v
                const float2 two_re = df_add(make_float2(cr.x, cr.y), make_float2(cr.x, cr.y));
                const cdf d0 = cdf_add(zv, make_float4(-two_re.x, -two_re.y, 0.f, 0.f));
                const cdf al = cdf_mul(tau, cdf_mul(cdf_conj(tau), d0));
                s_alpha = make_float4(-0.5f * al.x, -0.5f * al.y, -0.5f * al.z, -0.5f * al.w);
            }
        } else if (wid == 1) {   // W[k,l'], V[k,l'] (l' < l) and z_k of the current column's index k
            if (lane < l) {
                cwv[lane] = __ldcg(a.W + (size_t)lane * n + k);
                cwv[kNb + 1 + lane] = __ldcg(a.V + (size_t)lane * n + k);
            }
            if (lane == 0) {
                const cdf zr = __ldcg(a.zbuf + k), tk = __ldcg(a.zbuf + n + k);
                s_zk = s >= 0 ? cdf_fma(tk, inv, zr) : zr;
            }
        } else if (wid == 2) {   // z and v of own indices
            for (int m = m0 + lane; m < ncl; m += 32) {
                const int i = blk + m * G;
                if (s >= 0) {
                    zown[m] = cdf_fma(ztop[m], inv, zown[m]);
                    vown[m] = i == s + 1 ? make_float4(1.f, 0.f, 0.f, 0.f) : cdf_mul(Cs[i], inv);
                } else {
                    vown[m] = Cs[i];
                }
            }
        } else if (l == 0) {
            // first step of a panel: column k may have been updated by its owner's panel-end
            // update after phase 1 read it, so its entries are read again here
            for (int m = m0 + tid - 96; m < ncl; m += kTriThreads - 96) colk[m] = __ldcg(col(k) + blk + m * G);
        }
        __syncthreads();
        const cdf alpha = s_alpha;
        // own indices i > s: corr_i = sum_{l' < l} V[i,l'] s1_l' + W[i,l'] s2_l' (lanes over l'),
        // y_i = tau (z_i - corr_i), w_i = y_i + alpha v_i; column l of V and W.  The last warp
        // also forms W[k,l] = w_k of the current column's index (every CTA, redundantly).
        for (int t = wid; t < nown + 1; t += kTriWarps) {
            const bool own = t < nown;
            const int m = m0 + t;
            cdf c = cdf_zero();
            if (lane < l) {
                const cdf vi = own ? WVo(m, kNb + lane) : cwv[kNb + 1 + lane];
                const cdf wi = own ? WVo(m, lane) : cwv[lane];
                c = cdf_fma(cdf_mul(vi, s12[lane]), wi, s12[kNb + 1 + lane]);
            }
            c = cdf_warp_sum(c);
            if (lane == 0) {
                if (own) {
                    const cdf y = cdf_mul(tau, cdf_add(zown[m], cdf_neg(c)));
                    const cdf w = cdf_fma(y, alpha, vown[m]);
                    const int i = blk + m * G;
                    wown[m] = w;
                    WVo(m, l) = w;
                    WVo(m, kNb + l) = vown[m];
                    a.W[(size_t)l * n + i] = w;
                    a.V[(size_t)l * n + i] = vown[m];
                } else if (k <= n - 1) {
                    const cdf y = cdf_mul(tau, cdf_add(s_zk, cdf_neg(c)));
                    const cdf vk = s >= 0 ? make_float4(1.f, 0.f, 0.f, 0.f) : Cs[0];
                    cwv[l] = cdf_fma(y, alpha, vk);
                    cwv[kNb + 1 + l] = vk;
                }
            }
        }
        __syncthreads();
        // the current column k on own rows i >= k: A[i,k] - sum_{l' <= l} (V[i,l'] conj(W[k,l'])
        // + W[i,l'] conj(V[k,l'])) (lanes over l'), and its squared norm below row k + 1
        float nh = 0.f, nl = 0.f;
        for (int m = m0 + wid; m < ncl; m += kTriWarps) {
            const int i = blk + m * G;
            cdf t = cdf_zero();
            if (lane <= l)
                t = cdf_fma(cdf_mul(WVo(m, kNb + lane), cdf_conj(cwv[lane])), WVo(m, lane),
                            cdf_conj(cwv[kNb + 1 + lane]));
            t = cdf_warp_sum(t);
            if (lane == 0) {
                const cdf ai = cdf_add(colk[m], cdf_neg(t));
                a.ncol[i] = ai;
                if (i >= k + 2) {
                    df_acc(nh, nl, ai.x, ai.y, ai.x, ai.y);
                    df_acc(nh, nl, ai.z, ai.w, ai.z, ai.w);
                }
            }
        }
        if (lane == 0) s_nrm[wid] = df_fin(nh, nl);
        __syncthreads();
        if (tid == 0) {
            float2 t = s_nrm[0];
            for (int w = 1; w < kTriWarps; ++w) t = df_add(t, s_nrm[w]);
            a.npart[blk] = t;
        }
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;

        // ---------------- panel end: A -= V W^H + W V^H on own columns >= k, rows >= k ----------------
        if (!a.tc_update && l == kNb - 1 && s < n - 2) {
            const int nc = ncl - m0;
            for (int c0 = 0; c0 < nc; c0 += kHerCols) {
                const int cn = min(kHerCols, nc - c0);
                for (int r = k + tid; r < n; r += kTriThreads) {
                    float acc[kHerCols][4];
#pragma unroll
                    for (int c = 0; c < kHerCols; ++c) {
                        const cdf q = c < cn ? __ldcs(col(blk + (m0 + c0 + c) * G) + r) : cdf_zero();
                        acc[c][0] = q.x;
                        acc[c][1] = q.y;
                        acc[c][2] = q.z;
                        acc[c][3] = q.w;
                    }
                    cdf vn = __ldcg(a.V + r), wn = __ldcg(a.W + r);   // the next reflector's row, loaded ahead
                    for (int ll = 0; ll < kNb; ++ll) {
                        const cdf vr = vn, wr = wn;
                        if (ll + 1 < kNb) {
                            vn = __ldcg(a.V + (size_t)(ll + 1) * n + r);
                            wn = __ldcg(a.W + (size_t)(ll + 1) * n + r);
                        }
#pragma unroll
                        for (int c = 0; c < kHerCols; ++c) {
                            if (c >= cn) break;
                            const cdf wc = WVo(m0 + c0 + c, ll), vc = WVo(m0 + c0 + c, kNb + ll);
                            // acc -= vr conj(wc) + wr conj(vc)
                            df_acc(acc[c][0], acc[c][1], -vr.x, -vr.y, wc.x, wc.y);
                            df_acc(acc[c][0], acc[c][1], -vr.z, -vr.w, wc.z, wc.w);
                            df_acc(acc[c][0], acc[c][1], -wr.x, -wr.y, vc.x, vc.y);
                            df_acc(acc[c][0], acc[c][1], -wr.z, -wr.w, vc.z, vc.w);
                            df_acc(acc[c][2], acc[c][3], -vr.z, -vr.w, wc.x, wc.y);
                            df_acc(acc[c][2], acc[c][3], vr.x, vr.y, wc.z, wc.w);
                            df_acc(acc[c][2], acc[c][3], -wr.z, -wr.w, vc.x, vc.y);
                            df_acc(acc[c][2], acc[c][3], wr.x, wr.y, vc.z, vc.w);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < kHerCols; ++c) {
                        if (c >= cn) break;
                        const float2 re = df_fin(acc[c][0], acc[c][1]), im = df_fin(acc[c][2], acc[c][3]);
                        __stcs(col(blk + (m0 + c0 + c) * G) + r, make_float4(re.x, re.y, im.x, im.y));
                    }
                }
            }
            __syncthreads();
        }
    }
    if (a.s_end == n - 1 && blk == 0 && tid == 0) {
        const cdf z = __ldcg(a.ncol + (n - 1));
        a.d[n - 1] = df_to(make_float2(z.x, z.y));
    }
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
                                  float* d32, float* e2_32, float2* d_df, float2* e2_df, TriBounds* out) {
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
        e2_df[i] = df_from(e2[i]);
        if (small && (int)i + 1 < m) m = (int)i + 1;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        d32[i] = (float)d[i];
        d_df[i] = df_from(d[i]);
    }
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
    // the next row's operands are loaded a row ahead, off the recurrence's chain
    float dn = i0 + 1 < i1 ? __ldg(d + i0 + 1) : 0.f, en = i0 + 1 < i1 ? __ldg(e2 + i0) : 0.f;
    for (int i = i0 + 1; i < i1; ++i) {
        const float di = dn, ei = en;
        if (i + 1 < i1) {
            dn = __ldg(d + i + 1);
            en = __ldg(e2 + i);
        }
        q = (di - x) - ei / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.f;
    }
    return c;
}

// The same count in double-float on the FP32 pipe, from the three-term
// recurrence of the leading principal minors p_i = det(T[i0..i] - x),
//   p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}   (Sturm: sign changes count),
// which needs no division: two double-float multiply-adds per row.  p_i and
// p_{i-1} are rescaled together by an exact power of two whenever the larger
// leaves [2^-40, 2^40] (FP32's exponent range); an exact zero p_i becomes
// -2^-60 p_{i-1}, the tiny negative pivot of the ratio form.
__device__ __forceinline__ int sturm_count_df(const float2* __restrict__ d, const float2* __restrict__ e2, int i0,
                                              int i1, float2 x) {
    const float2 nx = df_neg(x);
    float2 pm = make_float2(1.f, 0.f);
    float2 p = df_add(__ldg(d + i0), nx);
    if (p.x == 0.f) p = make_float2(-0x1p-60f, 0.f);
    int c = p.x < 0.f;
    const float2 z = make_float2(0.f, 0.f);
    float2 dn = i0 + 1 < i1 ? __ldg(d + i0 + 1) : z, en = i0 + 1 < i1 ? __ldg(e2 + i0) : z;
    for (int i = i0 + 1; i < i1; ++i) {
        const float2 di = dn, ei = en;
        if (i + 1 < i1) {
            dn = __ldg(d + i + 1);
            en = __ldg(e2 + i);
        }
        const float2 dx = df_add(di, nx);
        float sh = 0.f, sl = 0.f;
        df_acc(sh, sl, dx.x, dx.y, p.x, p.y);
        df_acc(sh, sl, -ei.x, -ei.y, pm.x, pm.y);
        float2 pn = df_fin(sh, sl);
        if (pn.x == 0.f) pn = make_float2(-p.x * 0x1p-60f, 0.f);
        c += (pn.x < 0.f) != (p.x < 0.f);
        pm = p;
        p = pn;
        const float big = fmaxf(fabsf(p.x), fabsf(pm.x));
        if (big > 0x1p40f || big < 0x1p-40f) {
            const int ex = ((__float_as_int(big) >> 23) & 0xff) - 127;   // big = 1.f x 2^ex
            const float sc = __int_as_float((127 - ex) << 23);            // 2^-ex, exact
            p = make_float2(p.x * sc, p.y * sc);
            pm = make_float2(pm.x * sc, pm.y * sc);
        }
    }
    return c;
}

// S lanes per level: (S + 1)-section of the Gershgorin interval with Sturm
// counts: rounds in FP32 until the bracket is below 2 ||T|| / 1.2e6 (under the
// FP32 counts' backward error), the bracket widened by that error
// (16 eps_32 (||T|| + |x|)), then rounds in double-float until it has shrunk
// by 1.3e9 more, to about 1e-14 ||T||, below the backward error of the
// double-float reduction that made T.  Both kinds of count run on the FP32
// pipe.  With few levels the cost is each warp's chain of dependent
// instructions, so wide rounds (S = 32: 4 + 6 rounds) beat narrow ones; with
// thousands of levels the kernel is issue-bound and S = 8 (7 + 10 rounds, 136
// counts per level instead of 320) wins.  Every lane runs all rounds (uniform
// ballots).  Levels k < m belong to rows [0, m), the others to rows [m, n).
// Launched as blocks of four warps, one per SM sub-partition.
template <int S>
struct Sect {
    static constexpr unsigned mask = S == 32 ? 0xffffffffu : ((1u << (S & 31)) - 1u);
    static constexpr int rounds32 = S == 32 ? 4 : (S == 16 ? 5 : 7);   // (S + 1)^rounds32 >= 1.2e6
    static constexpr int rounds_df = S == 32 ? 6 : (S == 16 ? 8 : 10);  // (S + 1)^rounds_df >= 1.3e9
    static_assert(S == 8 || S == 16 || S == 32, "8-, 16- or 32-lane sections");
};
constexpr int kBisectThreads = 128;
constexpr int64_t kBisectNarrowFrom = 2048;   // levels from which the 9-section beats the 33-section
template <int S>
__global__ void __launch_bounds__(kBisectThreads) bisect_kernel(const float2* __restrict__ d_df,
                                                                const float2* __restrict__ e2_df,
                                                                const float* __restrict__ d32,
                                                                const float* __restrict__ e2_32, int64_t n,
                                                                const TriBounds* __restrict__ bnd, double* lam) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, sub = lane % S, base = lane - sub;
    const int64_t k = min(t / S, n - 1);
    const TriBounds b = *bnd;
    const int i0 = k < b.m ? 0 : b.m, i1 = k < b.m ? b.m : (int)n;
    const int kk = (int)(k - i0);
    float lof = (float)b.gl, hif = (float)b.gu;
    for (int it = 0; it < Sect<S>::rounds32; ++it) {
        const float x = lof + (hif - lof) * (float)(sub + 1) * (1.0f / (S + 1));
        const int c = sturm_count32(d32, e2_32, i0, i1, x, b.pivmin32);
        const unsigned q = (__ballot_sync(0xffffffffu, c > kk) >> base) & Sect<S>::mask;
        const int ls = q ? __ffs(q) - 1 : S;   // first point above level kk
        const float xl = __shfl_sync(0xffffffffu, x, base + (ls > 0 ? ls - 1 : 0));
        const float xh = __shfl_sync(0xffffffffu, x, base + (ls < S ? ls : S - 1));
        if (ls > 0) lof = xl;
        if (ls < S) hif = xh;
    }
    const double del = 16.0 * FLT_EPSILON * (b.tnorm + fmax(fabs((double)lof), fabs((double)hif)));
    double lo = fmax(b.gl, (double)lof - del), hi = fmin(b.gu, (double)hif + del);
    for (int it = 0; it < Sect<S>::rounds_df; ++it) {
        const double x = lo + (hi - lo) * (double)(sub + 1) * (1.0 / (S + 1));
        const int c = sturm_count_df(d_df, e2_df, i0, i1, df_from(x));
        const unsigned q = (__ballot_sync(0xffffffffu, c > kk) >> base) & Sect<S>::mask;
        const int ls = q ? __ffs(q) - 1 : S;   // first point above level kk
        const double xl = __shfl_sync(0xffffffffu, x, base + (ls > 0 ? ls - 1 : 0));
        const double xh = __shfl_sync(0xffffffffu, x, base + (ls < S ? ls : S - 1));
        if (ls > 0) lo = xl;
        if (ls < S) hi = xh;
    }
    if (sub == 0 && t / S < n) lam[k] = 0.5 * (lo + hi);
}

// Squared first component of the eigenvector of rows [0, m) for level k < m,
// from the twisted factorisation T - lam = N_r Delta_r N_r^T at the twist
// index r with the smallest |gamma_r| (gamma_r = D+_r + D-_r - (d_r - lam));
// zero for levels of rows [m, n).  With z_r = 1, z_i = -L+_i z_{i+1} above r
// and z_{i+1} = -U-_i z_i below it, so
//   z_0^2 = prod_{i<r} L+_i^2,  sum_{i<r} z_i^2 = h_r,  sum_{i>r} z_i^2 = t_r
// with L+_i^2 = e_i^2 / (D+_i)^2, h_{i+1} = L+_i^2 (1 + h_i),
// U-_i^2 = e_i^2 / (D-_{i+1})^2 and t_i = U-_i^2 (1 + t_{i+1}).
// A block of two warps takes 32 levels (one per lane).  The pivots D+ (warp
// 0, top-down) and D- (warp 1, bottom-up) follow the ratio recurrences
// D_next = (d - lam) - e^2 / D in double-float on the FP32 pipe and are
// stored; both warps then scan half of the twist indices; last, warp 0
// forms z_0^2 and h_r from the stored D+ above r and warp 1 t_r from the D-
// below it, in FP64 (these products can leave FP32's range), with the
// factors e^2 / D^2 formed in double-float unless |D| < 2^-50.
// st: scratch of 2 [m][n] double-float arrays (level index fastest).
__device__ __forceinline__ float2 twist_clamp(float2 p, float piv) {
    return fabsf(p.x) < piv ? make_float2(-piv, 0.f) : p;
}
// e^2 / D^2 as a double (D clamped, nonzero)
__device__ __forceinline__ double twist_factor(float2 e2, float2 D, double e2d) {
    if (fabsf(D.x) >= 0x1p-50f) {
        const float2 r = df_rcp(D);
        return df_to(df_mul(e2, df_mul(r, r)));
    }
    const double Dd = df_to(D);
    return e2d / (Dd * Dd);
}
__global__ void __launch_bounds__(64) twisted_weights_kernel(const float2* __restrict__ d_df,
                                                             const float2* __restrict__ e2_df,
                                                             const double* __restrict__ e2d, int64_t n,
                                                             const TriBounds* __restrict__ bnd,
                                                             const double* __restrict__ lam, float2* st, double* w) {
    __shared__ float s_best[2][32];
    __shared__ int s_r[2][32];
    __shared__ double s_t[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * 32 + lane;
    const TriBounds b = *bnd;
    const int m = b.m;
    const bool act = k0 < m;
    const int64_t k = act ? k0 : 0;
    const float2 nl = df_neg(df_from(lam[k]));
    const float piv = b.pivmin32;
    float2* Dp = st;
    float2* Dm = st + (size_t)n * n;
    if (act) {
        if (wid == 0) {   // top-down: D+_i (clamped)
            float2 p = twist_clamp(df_add(__ldg(d_df), nl), piv);
            float2 en = m > 1 ? __ldg(e2_df) : make_float2(0.f, 0.f), dn = m > 1 ? __ldg(d_df + 1) : en;
            for (int i = 0; i + 1 < m; ++i) {
                const float2 ei = en, di = dn;   // operands of this row, the next row's loaded ahead
                if (i + 2 < m) {
                    en = __ldg(e2_df + i + 1);
                    dn = __ldg(d_df + i + 2);
                }
                Dp[(size_t)i * n + k] = p;
                const float2 t = df_mul(ei, df_rcp(p));
                const float2 dx = df_add(di, nl);
                p = twist_clamp(fabsf(t.x) < 0x1p120f ? df_add(dx, df_neg(t)) : make_float2(-t.x, 0.f), piv);
            }
            Dp[(size_t)(m - 1) * n + k] = p;
        } else {          // bottom-up: D-_i (as computed, clamped where used)
            float2 q = df_add(__ldg(d_df + m - 1), nl);
            Dm[(size_t)(m - 1) * n + k] = q;
            float2 en = m > 1 ? __ldg(e2_df + m - 2) : make_float2(0.f, 0.f), dn = m > 1 ? __ldg(d_df + m - 2) : en;
            for (int i = m - 2; i >= 0; --i) {
                const float2 ei = en, di = dn;
                if (i > 0) {
                    en = __ldg(e2_df + i - 1);
                    dn = __ldg(d_df + i - 1);
                }
                const float2 t = df_mul(ei, df_rcp(twist_clamp(q, piv)));
                const float2 dx = df_add(di, nl);
                q = fabsf(t.x) < 0x1p120f ? df_add(dx, df_neg(t)) : make_float2(-t.x, 0.f);
                Dm[(size_t)i * n + k] = q;
            }
        }
    }
    __syncthreads();
    // twist index: smallest |gamma_i| over this warp's half (ties: lowest i)
    float best = INFINITY;
    int rb = 0;
    if (act) {
        const int h0 = wid == 0 ? 0 : m / 2, h1 = wid == 0 ? m / 2 : m;
        // unrolled so that the loads of several rows are in flight at once (the stored
        // factors come from DRAM and one warp per SM sub-partition cannot hide that latency)
#pragma unroll 8
        for (int i = h0; i < h1; ++i) {
            const float2 g = df_add(df_add(Dp[(size_t)i * n + k], Dm[(size_t)i * n + k]),
                                    df_neg(df_add(__ldg(d_df + i), nl)));
            const float ga = fabsf(g.x);
            if (ga < best) {
                best = ga;
                rb = i;
            }
        }
    }
    s_best[wid][lane] = best;
    s_r[wid][lane] = rb;
    __syncthreads();
    const int r = s_best[1][lane] < s_best[0][lane] ? s_r[1][lane] : s_r[0][lane];
    double P = 1.0, h = 0.0, t = 0.0;
    if (act) {
        if (wid == 0) {
#pragma unroll 8
            for (int i = 0; i < r; ++i) {
                const double L2 = twist_factor(__ldg(e2_df + i), Dp[(size_t)i * n + k], __ldg(e2d + i));
                P *= L2;
                h = fma(L2, h, L2);
            }
        } else {
#pragma unroll 8
            for (int i = m - 2; i >= r; --i) {
                const double U2 = twist_factor(__ldg(e2_df + i), twist_clamp(Dm[(size_t)(i + 1) * n + k], piv),
                                               __ldg(e2d + i));
                t = U2 * (1.0 + t);
            }
            s_t[lane] = t;
        }
    }
    __syncthreads();
    if (wid == 0 && act) {
        w[k] = P * rcp_nr(1.0 + h + s_t[lane]);
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
    // order-preserving integer keys of the (finite) levels: the comparisons
    // run on the integer pipe instead of GB300's narrow FP64 pipe
    auto key = [](double v) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    };
    const double x = lam[k];
    const unsigned long long kx = key(x);
    int64_t pos = 0;
    for (int64_t j = 0; j < n; ++j) {
        const unsigned long long ky = key(__ldg(lam + j));
        pos += (ky < kx) || (ky == kx && j < k);
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
    // v0 n, ncol 2n, xbuf 2n, spart 2 x 1024 (16 bytes each); d, e, e2, lam, w (n doubles); d32, e2_32 (n floats);
    // d_df, e2_df (n float2); twisted pivots 2 n*n float2; the blocked reduction's V and W (2 kNb n,
    // 16 bytes each), its norm parts (1024 float2) and s dots (2 kNb); 256-byte alignment of each piece
    return sizeof(double2) * (size_t)(5 * n + 2048) + sizeof(double) * (size_t)(5 * n) +
           sizeof(float2) * (size_t)(2 * n * n) + sizeof(float) * (size_t)(2 * n) + sizeof(float2) * (size_t)(2 * n) +
           sizeof(cdf) * (size_t)(2 * kNb * n + 4 * kNb) + sizeof(float2) * 1024 + panel_update_tc_bytes(n) +
           tridiag2_bytes(n) + 16384;
}

// the blocked reduction keeps a column (16 n bytes) and the panel coefficients
// of its own columns in 227 KB of shared memory: n up to about 10 000
int tridiag_max_dim() { return 8192; }

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
                            double* osc, double* wsum, int* err, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                            long wait_polls, int variant, int* used) {
    if (n < 1 || n > tridiag_max_dim()) return fail(BSE_EUNSUPPORTED, "tridiagonal path: n = %lld", (long long)n);
    char* p = (char*)scratch;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)q;
    };
    double2* v0 = (double2*)take(sizeof(double2) * n);
    cdf* ncol = (cdf*)take(sizeof(cdf) * 2 * n);
    cdf* xbuf = (cdf*)take(sizeof(cdf) * 2 * n);
    cdf* spart = (cdf*)take(sizeof(cdf) * 2048);
    double* d = (double*)take(sizeof(double) * n);
    double* e = (double*)take(sizeof(double) * n);
    double* e2 = (double*)take(sizeof(double) * n);
    float* d32 = (float*)take(sizeof(float) * n);
    float* e2_32 = (float*)take(sizeof(float) * n);
    float2* d_df = (float2*)take(sizeof(float2) * n);
    float2* e2_df = (float2*)take(sizeof(float2) * n);
    double* lam = (double*)take(sizeof(double) * n);
    double* w = (double*)take(sizeof(double) * n);
    double* beta0 = (double*)take(sizeof(double));
    TriBounds* bnd = (TriBounds*)take(sizeof(TriBounds));
    unsigned* bar = (unsigned*)take(sizeof(unsigned));
    float2* dp = (float2*)take(sizeof(float2) * 2 * n * n);
    cdf* Vp = (cdf*)take(sizeof(cdf) * kNb * n);
    cdf* Wp = (cdf*)take(sizeof(cdf) * kNb * n);
    cdf* sdot = (cdf*)take(sizeof(cdf) * 4 * kNb);
    float2* npart = (float2*)take(sizeof(float2) * 1024);
    void* tcs = take(panel_update_tc_bytes(n));
    void* two = take(tridiag2_bytes(n));

    int dev = 0, sms = 0, maxsm = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BSE_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int G = (int)std::min<int64_t>(sms, std::max<int64_t>(1, (n + 3) / 4));
    const size_t static_smem = sizeof(cdf) * (kTriWarps + 3) + 64;
    const size_t vec_bytes = sizeof(cdf) * 3 * (size_t)n;   // v, w and the next column of a step
    const size_t cols_bytes = sizeof(cdf) * (size_t)((n - 1) / G + 1) * n;
    const bool smem = variant == 0 && vec_bytes + cols_bytes + static_smem <= (size_t)maxsm;
    // above the shared-memory size: the blocked reduction up to n = 1800, where the two-stage
    // one (whose band-to-tridiagonal stage takes about 9 us per row) overtakes it
    if (variant == 0 && !smem && n >= kTwoStageFrom) variant = 3;
    const bool tcu = variant != 2;   // blocked: panel-end update on the tensor cores between launches
    if (!smem) G = (int)std::min<int64_t>(sms, n);
    if (!smem && tri_blocked_smem(n, G) > (size_t)maxsm)
        return fail(BSE_EUNSUPPORTED, "tridiagonal path: n = %lld exceeds shared memory", (long long)n);
    if (used) *used = variant == 3 ? 3 : (smem ? 0 : (tcu ? 1 : 2));

    BSE_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    BSE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    BSE_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, st));
    reflect0_kernel<<<1, kTriThreads, 0, st>>>(b, n, v0, beta0);
    note_launch();
    BSE_CUDA(cudaGetLastError());

    if (variant == 3) {   // two-stage: dense -> band -> tridiagonal
        if (ev0) BSE_CUDA(cudaEventRecord(ev0, st));
        BSE_TRY(launch_tridiag2(reinterpret_cast<cdf*>(h), n, v0, beta0, d, e, Vp, Wp, tcs, two, err, st, wait_polls));
        if (ev1) BSE_CUDA(cudaEventRecord(ev1, st));
    } else if (smem) {
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
        a.spin = wait_limit(wait_polls, kGridSpinLimit);
        void* args[] = {&a};
        const size_t dyn = vec_bytes + cols_bytes;
        const void* fn = (const void*)tridiag_kernel<true>;
        BSE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        int per_sm = 0;
        BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTriThreads, dyn));
        if (per_sm < 1 || G > per_sm * sms) return fail(BSE_EUNSUPPORTED, "tridiagonal kernel cannot be co-resident");
        if (ev0) BSE_CUDA(cudaEventRecord(ev0, st));
        BSE_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kTriThreads), args, dyn, st));
        note_launch();
        if (ev1) BSE_CUDA(cudaEventRecord(ev1, st));
    } else {
        TriBArgs a;
        a.A = reinterpret_cast<cdf*>(h);
        a.n = n;
        a.v0 = v0;
        a.beta0 = beta0;
        a.V = Vp;
        a.W = Wp;
        a.ncol = ncol;
        a.npart = npart;
        a.zbuf = xbuf;
        a.zpart = spart;
        a.sdot = sdot;
        a.d = d;
        a.e = e;
        a.bar = bar;
        a.err = err;
        a.spin = wait_limit(wait_polls, kGridSpinLimit);
        // the last columns, about 80 MB of them, stay in L2 between steps (the other columns and
        // the panel's vectors share the rest); a block that fits keeps all its columns there
        const int64_t keep = std::min<int64_t>(n, (int64_t)80000000 / (16 * n));
        a.resident_from = (int)(n - keep);
        // three stages of up to 256 rows per warp in the shared memory left over
        const size_t base_smem = tri_blocked_smem(n, G);
        const int64_t room = ((int64_t)maxsm - (int64_t)base_smem - 1024) / (kTriWarps * 3 * (int64_t)sizeof(cdf));
        a.stage_rows = room >= 64 ? (int)std::min<int64_t>(256, room / 32 * 32) : 0;
        void* args[] = {&a};
        const size_t dyn = base_smem + (size_t)kTriWarps * 3 * a.stage_rows * sizeof(cdf);
        const void* fn = (const void*)tridiag_blocked_kernel;
        BSE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        int per_sm = 0;
        BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTriThreads, dyn));
        if (per_sm < 1 || G > per_sm * sms) return fail(BSE_EUNSUPPORTED, "tridiagonal kernel cannot be co-resident");
        if (ev0) BSE_CUDA(cudaEventRecord(ev0, st));
        // with the tensor-core update one launch per panel (steps s0 .. s0 + kNb - 1), each
        // followed by the panel-end update of the trailing block from k = s0 + kNb on
        const int64_t span = tcu ? kNb : n;
        for (int64_t s0 = -1; s0 < n - 1; s0 += span) {
            const int64_t s1 = std::min<int64_t>(s0 + span, n - 1);
            if (s0 > -1) BSE_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
            a.s_begin = (int)s0;
            a.s_end = (int)s1;
            a.tc_update = tcu ? 1 : 0;
            BSE_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kTriThreads), args, dyn, st));
            note_launch();
            if (tcu && s1 <= n - 2)
                BSE_TRY(launch_panel_update_tc(a.A, n, (int)s1, a.resident_from, Vp, Wp, tcs, err, st, wait_polls));
        }
        if (ev1) BSE_CUDA(cudaEventRecord(ev1, st));
    }

    tri_bounds_kernel<<<1, kTriThreads, 0, st>>>(d, e, n, e2, d32, e2_32, d_df, e2_df, bnd);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    if (n >= kBisectNarrowFrom)
        bisect_kernel<8><<<(unsigned)((8 * n + kBisectThreads - 1) / kBisectThreads), kBisectThreads, 0, st>>>(
            d_df, e2_df, d32, e2_32, n, bnd, lam);
    else
        bisect_kernel<32><<<(unsigned)((32 * n + kBisectThreads - 1) / kBisectThreads), kBisectThreads, 0, st>>>(
            d_df, e2_df, d32, e2_32, n, bnd, lam);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    twisted_weights_kernel<<<(unsigned)((n + 31) / 32), 64, 0, st>>>(d_df, e2_df, e2, n, bnd, lam, dp, w);
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
