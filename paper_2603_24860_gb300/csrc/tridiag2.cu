// Two-stage reduction of a Hermitian block to a real tridiagonal T that keeps
// e_0 fixed (sm_103a): the stage that feeds the eigenvector-free spectrum
// (Eqs. oscillator, oscillatorA; levels from T, weights from the first
// components of its eigenvectors).
//
// The start reflector H0 (which maps conj(U^T B) onto e_0) is applied to the
// whole block first.  Then
//
//   stage 1  dense -> band of half-bandwidth 32.  Panel j holds the columns
//            c0 = 32 j .. c0 + 31 and the rows r1 = c0 + 32 .. n - 1 below the
//            band.  Its Householder QR (zlarfg reflectors on rows >= r1, so
//            that e_0 stays fixed) gives Q = I - V T V^H (compact WY form, T by
//            the forward column-wise recurrence) and leaves [R; 0] in the
//            panel.  The trailing block A22 = A[r1:, r1:] becomes Q^H A22 Q =
//            A22 - V W^H - W V^H with Y = A22 V T and W = Y - 1/2 V (T^H V^H Y):
//            one pass of A22 through a GEMM for A22 V (double-float on the
//            CUDA cores, split over K) and the rank-64 update on the tensor
//            cores (her2k_tc.cu).  The trailing block is read twice per panel
//            instead of once per reflection step.
//   stage 2  band -> tridiagonal by bulge chasing.  Sweep i annihilates column
//            i below the subdiagonal with a reflector on rows i+1 .. i+32 and
//            chases the bulge down the band in windows of 32 rows: task t of
//            sweep i reflects the first column of the block left by task t-1,
//            applies the reflector to the rest of that block (left), to the
//            32 x 32 diagonal block (both sides) and to the block below
//            (right), which becomes the next bulge.  One CTA runs a sweep at a
//            time; sweep i may load the window of task t but its last column
//            once sweep i - 1 is done with those entries, and the last column
//            (33 entries) once sweep i - 1 has published the critical part of
//            its task t + 1; the left block needs no wait.  Only the lower
//            triangle of the band is read and written.
//
// Every reflector acts on rows >= 1, so Q e_0 = e_0.  The tridiagonal matrix
// left in the band is complex Hermitian; a diagonal unitary scaling makes its
// off-diagonal real and non-negative without changing the levels or the
// magnitudes of the first eigenvector components: d_i = Re A[i,i],
// e_i = |A[i+1,i]|.  All arithmetic is double-float (dfloat.h) on the FP32
// pipe, the rank-64 update excepted (exact bf16 digit products).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "dfloat.h"
#include "fp64_fast.h"
#include "grid_sync.h"
#include "internal.h"
#include "reflector.h"

namespace bse {

namespace {

constexpr int kB = 32;              // half-bandwidth of stage 1 = reflectors per panel
constexpr int kT2 = 256;            // threads of most kernels here
constexpr int kW2 = kT2 / 32;
constexpr int kMaxKs = 8;           // K splits of the A22 V product (at least those of zgemm_tc.cu)
constexpr int kQrMaxCta = 32;       // CTAs of the panel QR
constexpr int kGramRows = 32;       // rows per CTA of the 32 x 32 Gram products
constexpr int kSweepDone = 1 << 30;

__device__ __forceinline__ cdf conjc(cdf a) { return make_float4(a.x, a.y, -a.z, -a.w); }
__device__ __forceinline__ cdf negc(cdf a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ cdf onec() { return make_float4(1.f, 0.f, 0.f, 0.f); }

// raw double-float complex accumulator (s, lo per part), normalised at the end
struct CAcc {
    float sr, lr, si, li;
    __device__ __forceinline__ void zero() { sr = lr = si = li = 0.f; }
    // += a b
    __device__ __forceinline__ void mac(cdf a, cdf b) {
        df_acc(sr, lr, a.x, a.y, b.x, b.y);
        df_acc(sr, lr, -a.z, -a.w, b.z, b.w);
        df_acc(si, li, a.x, a.y, b.z, b.w);
        df_acc(si, li, a.z, a.w, b.x, b.y);
    }
    // += conj(a) b
    __device__ __forceinline__ void dot(cdf a, cdf b) {
        df_acc(sr, lr, a.x, a.y, b.x, b.y);
        df_acc(sr, lr, a.z, a.w, b.z, b.w);
        df_acc(si, li, a.x, a.y, b.z, b.w);
        df_acc(si, li, -a.z, -a.w, b.x, b.y);
    }
    __device__ __forceinline__ cdf get() const {
        const float2 r = df_fin(sr, lr), i = df_fin(si, li);
        return make_float4(r.x, r.y, i.x, i.y);
    }
};

__device__ __forceinline__ float2 warp_sum_df(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    return v;
}

// sum of a raw accumulator over the G lanes of a group (lanes G g .. G g + G - 1): per
// level TwoSum of the leading words, the low words and TwoSum's error added (the error
// model of cdf_add), normalised once at the end
template <int G>
__device__ __forceinline__ cdf cacc_group_sum(CAcc a) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        const float sr = __shfl_xor_sync(0xffffffffu, a.sr, o), lr = __shfl_xor_sync(0xffffffffu, a.lr, o);
        const float si = __shfl_xor_sync(0xffffffffu, a.si, o), li = __shfl_xor_sync(0xffffffffu, a.li, o);
        float er, ei;
        two_sum(a.sr, sr, a.sr, er);
        two_sum(a.si, si, a.si, ei);
        a.lr = __fadd_rn(a.lr, __fadd_rn(lr, er));
        a.li = __fadd_rn(a.li, __fadd_rn(li, ei));
    }
    return a.get();
}
__device__ __forceinline__ cdf cacc_warp_sum(CAcc a) { return cacc_group_sum<32>(a); }

// the block in place from FP64 to double-float (16 bytes per element either way)
__global__ void to_cdf_kernel(cdf* A, int64_t nn) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nn; k += (int64_t)gridDim.x * blockDim.x) {
        const double2 z = reinterpret_cast<const double2*>(A)[k];
        A[k] = cdf_from(z);
    }
}

// ---------------------------------------------------------------------------
// Start reflector H0 = I - beta v v^H (beta real): A <- H0 A H0 = A - v w^H - w v^H
// with y = A v, mu = v^H y (real) and w = beta y - beta^2 mu / 2 v.
// ---------------------------------------------------------------------------

// y_i = (A v)_i = sum_r conj(A[r,i]) v_r (A Hermitian): one warp per column
__global__ void h0_matvec_kernel(const cdf* __restrict__ A, int n, const double2* __restrict__ v0, cdf* y) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    const cdf* col = A + (size_t)i * n;
    CAcc acc;
    acc.zero();
    for (int r = lane; r < n; r += 32) acc.dot(__ldcg(col + r), cdf_from(v0[r]));
    cdf s = cdf_warp_sum(acc.get());
    if (lane == 0) y[i] = s;
}

// v and w as double-float vectors (one block).  H0 is unchanged by v -> v / |v|,
// beta -> beta |v|^2, which keeps every product in range whatever the size of the start
// vector (a nearly dark block has |v| of rounding size and beta ~ 1 / |v|^2); then
// mu = v^H y and w = beta y - beta^2 mu / 2 v with y = A v scaled the same way.
__global__ void h0_vectors_kernel(const double2* __restrict__ v0, const double* __restrict__ beta0, const cdf* y,
                                  int n, cdf* v, cdf* w) {
    __shared__ double s_d[kW2];
    __shared__ float2 s_part[kW2];
    __shared__ float2 s_c, s_b;
    __shared__ double s_sv;
    const int tid = threadIdx.x;
    double nv = 0.0;
    for (int r = tid; r < n; r += blockDim.x) nv += v0[r].x * v0[r].x + v0[r].y * v0[r].y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
    if ((tid & 31) == 0) s_d[tid >> 5] = nv;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_d[k];
        s_sv = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
        s_b = df_from(*beta0 * t);   // beta |v|^2
    }
    __syncthreads();
    const double sv = s_sv;
    float s = 0.f, lo = 0.f;
    for (int r = tid; r < n; r += blockDim.x) {
        const cdf a = cdf_from(make_double2(v0[r].x * sv, v0[r].y * sv)), b = y[r];
        const float2 br = df_mul(make_float2(b.x, b.y), df_from(sv)), bi = df_mul(make_float2(b.z, b.w), df_from(sv));
        df_acc(s, lo, a.x, a.y, br.x, br.y);   // Re(conj(a) b)
        df_acc(s, lo, a.z, a.w, bi.x, bi.y);
    }
    float2 t = warp_sum_df(df_fin(s, lo));
    if ((tid & 31) == 0) s_part[tid >> 5] = t;
    __syncthreads();
    if (tid == 0) {
        float2 mu = s_part[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) mu = df_add(mu, s_part[k]);
        const float2 b = s_b;
        s_c = df_mul(df_mul(df_mul(b, b), mu), make_float2(0.5f, 0.f));   // beta^2 mu / 2
    }
    __syncthreads();
    const float2 b = s_b, c = s_c, svf = df_from(sv);
    for (int r = tid; r < n; r += blockDim.x) {
        const cdf a = cdf_from(make_double2(v0[r].x * sv, v0[r].y * sv)), yy = y[r];
        v[r] = a;
        const float2 yr = df_mul(make_float2(yy.x, yy.y), svf), yi = df_mul(make_float2(yy.z, yy.w), svf);
        const float2 wr = df_add(df_mul(b, yr), df_neg(df_mul(c, make_float2(a.x, a.y))));
        const float2 wi = df_add(df_mul(b, yi), df_neg(df_mul(c, make_float2(a.z, a.w))));
        w[r] = make_float4(wr.x, wr.y, wi.x, wi.y);
    }
}

// A[r,i] -= v_r conj(w_i) + w_r conj(v_i) on the whole block
__global__ void rank2_all_kernel(cdf* A, int n, const cdf* __restrict__ v, const cdf* __restrict__ w) {
    const int64_t nn = (int64_t)n * n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nn; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / n), r = (int)(k - (int64_t)i * n);
        A[k] = cdf_rank2(A[k], v[r], w[r], w[i], v[i]);
    }
}

// ---------------------------------------------------------------------------
// Panel QR (cooperative; CTA b holds the panel rows rho in [b ch, (b+1) ch),
// one thread per row, in shared memory).  Per reflector l: the partial squared
// norms of column l below row l and its pivot; grid barrier; every CTA forms
// the reflector (zlarfg, v_l = 1) from the sums, scales its rows of v and adds
// its part of w = v^H P for the columns right of l; grid barrier; every CTA
// sums w and applies P <- P - conj(tau) v w to its rows.
// ---------------------------------------------------------------------------
struct PanelArgs {
    cdf* A;            // n x n, column-major, double-float
    int n, c0, r1, m;  // panel columns c0 .. c0 + 31, rows r1 .. r1 + m - 1 (r1 = c0 + 32)
    int nref;          // reflectors (min(32, m - 1))
    cdf* V;            // [32][n] reflector l at V[l n + r], zero above its row r1 + l
    cdf* tau;          // [32]
    float2* part;      // [G] partial squared norms
    cdf* piv;          // [32] pivots (entry l of column l after reflectors < l)
    cdf* wpart;        // [G][64] partial w (columns > l) and partial V^H v_l (entries 32 + k, k < l)
    cdf* T;            // [32][32] the T factor of Q = I - V T V^H (written by CTA 0)
    unsigned* bar;     // zero on entry
    int* err;
    long spin;
};

__global__ void __launch_bounds__(kT2, 1) panel_qr_kernel(PanelArgs a) {
    extern __shared__ __align__(16) cdf s_qr[];   // P rows: [32][ch], then V rows: [32][ch]
    __shared__ float2 s_red[kW2];
    __shared__ cdf s_w[2 * kB];
    __shared__ cdf s_T[kB][kB + 1];   // CTA 0: the T factor, column by column
    __shared__ cdf s_tau, s_inv;
    __shared__ float2 s_beta;
    __shared__ int s_flag;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int ch = (a.m + G - 1) / G;
    const int rho0 = b * ch, nown = max(0, min(a.m, rho0 + ch) - rho0);
    cdf* P = s_qr;                       // P[l * ch + t]
    cdf* Vs = s_qr + (size_t)kB * ch;    // Vs[l * ch + t]
    const int n = a.n;
    const int rho = rho0 + tid;          // this thread's panel row (tid < nown)
    const bool mine = tid < nown;
    for (int l = 0; l < kB; ++l) {
        const cdf x = mine ? __ldcg(a.A + (size_t)(a.c0 + l) * n + a.r1 + rho) : cdf_zero();
        if (tid < ch) {
            P[l * ch + tid] = x;
            Vs[l * ch + tid] = cdf_zero();
        }
    }
    __syncthreads();
    unsigned nbar = 0;
    for (int l = 0; l < a.nref; ++l) {
        // squared norm of column l below row l, and its pivot
        float s = 0.f, lo = 0.f;
        if (mine && rho > l) {
            const cdf x = P[l * ch + tid];
            df_acc(s, lo, x.x, x.y, x.x, x.y);
            df_acc(s, lo, x.z, x.w, x.z, x.w);
        }
        if (mine && rho == l) a.piv[l] = P[l * ch + tid];
        float2 t = warp_sum_df(df_fin(s, lo));
        if (lane == 0) s_red[wid] = t;
        __syncthreads();
        if (tid == 0) {
            for (int k = 1; k < kW2; ++k) t = df_add(t, s_red[k]);
            a.part[b] = t;
        }
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;
        // the reflector from the sums (warp 0), v on own rows, partial w = v^H P
        if (wid == 0) {
            float2 sg = make_float2(0.f, 0.f);
            for (int k = lane; k < G; k += 32) sg = df_add(sg, __ldcg(a.part + k));
            sg = warp_sum_df(sg);
            if (lane == 0) {
                cdf tau, inv;
                float2 beta;
                reflector(__ldcg(a.piv + l), sg, tau, inv, beta);
                s_tau = tau;
                s_inv = inv;
                s_beta = beta;
                if (b == 0) a.tau[l] = tau;
            }
        }
        __syncthreads();
        const cdf inv = s_inv;
        if (mine && rho >= l) {
            const cdf x = P[l * ch + tid];
            const cdf v = rho == l ? onec() : cdf_mul(x, inv);
            Vs[l * ch + tid] = v;
            P[l * ch + tid] = rho == l ? make_float4(s_beta.x, s_beta.y, 0.f, 0.f) : cdf_zero();
        }
        __syncthreads();
        // a warp per task, lanes over own rows: w_c = v^H P[:, c] (c > l) and
        // g_k = v_k^H v (k < l, for the T factor)
        for (int c = wid; c < kB - 1; c += kW2) {
            const int col = c < l ? c : c + 1;   // tasks: g_0 .. g_{l-1}, then w_{l+1} .. w_31
            const bool isg = c < l;
            CAcc acc;
            acc.zero();
            for (int u = lane; u < nown; u += 32)
                if (rho0 + u >= l) {
                    if (isg)
                        acc.dot(Vs[col * ch + u], Vs[l * ch + u]);
                    else
                        acc.dot(Vs[l * ch + u], P[col * ch + u]);
                }
            const cdf sum = cdf_warp_sum(acc.get());
            if (lane == 0) a.wpart[(size_t)b * 2 * kB + (isg ? kB + col : col)] = sum;
        }
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;
        // sums over the CTAs (four threads per entry); P <- P - conj(tau) v w on own rows >= l,
        // columns > l; CTA 0: column l of T, T[0:l, l] = -tau_l T[0:l, 0:l] g
        {
            const int ent = tid >> 2, k0 = tid & 3;
            const bool need = ent < kB ? ent > l : ent - kB < l;
            cdf sum = cdf_zero();
            if (need)
#pragma unroll 4
                for (int k = k0; k < G; k += 4) sum = cdf_add(sum, __ldcg(a.wpart + (size_t)k * 2 * kB + ent));
            sum = cdf_add(sum, cdf_shfl_xor(sum, 1));
            sum = cdf_add(sum, cdf_shfl_xor(sum, 2));
            if (k0 == 0 && need) s_w[ent] = sum;
        }
        __syncthreads();
        if (b == 0 && tid <= l) {
            if (tid == l) {
                s_T[l][l] = s_tau;
            } else {
                CAcc acc;
                acc.zero();
                for (int k = tid; k < l; ++k) acc.mac(s_T[tid][k], s_w[kB + k]);
                s_T[tid][l] = cdf_mul(negc(s_tau), acc.get());
            }
        }
        if (mine && rho >= l) {
            const cdf f = cdf_mul(conjc(s_tau), Vs[l * ch + tid]);   // conj(tau) v_rho
            for (int c = l + 1; c < kB; ++c) P[c * ch + tid] = cdf_fma(P[c * ch + tid], negc(f), s_w[c]);
        }
        __syncthreads();
    }
    // the panel ([R; 0]), the reflectors and T back to global memory
    if (b == 0)
        for (int e = tid; e < kB * kB; e += kT2) {
            const int r = e >> 5, c = e & 31;
            a.T[e] = r <= c && c < a.nref ? s_T[r][c] : cdf_zero();
        }
    if (mine)
        for (int l = 0; l < kB; ++l) {
            a.A[(size_t)(a.c0 + l) * n + a.r1 + rho] = P[l * ch + tid];
            a.V[(size_t)l * n + a.r1 + rho] = Vs[l * ch + tid];
        }
}

// ---------------------------------------------------------------------------
// The same panel QR on one thread-block cluster: the panel rows are spread over
// the cluster's CTAs (in shared memory, v_l stored in place of the entries it
// annihilates, beta_l on the diagonal), and the per-reflector sums travel through
// distributed shared memory with one cluster barrier per reflector instead of
// grid barriers and global-memory round trips.  A CTA reads another CTA's part
// only between the barrier after which it was written and the next one, and a
// final barrier keeps every CTA resident until the last remote read.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// the address of the same shared variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_rank(const void* p, uint32_t rank) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(ra)
                 : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return ra;
}
__device__ __forceinline__ cdf ld_cluster_cdf(uint32_t ra) {
    cdf v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(ra)
                 : "memory");
    return v;
}

// One cluster barrier per reflector.  Before reflector l is known, every CTA sums over
// its rows rho > l: sigma = |P[rho][l]|^2, d_c = conj(P[rho][l]) P[rho][c] (c > l) and
// h_k = conj(v_k[rho]) P[rho][l] (k < l); the owner of row l adds the pivot row P[l][c]
// (c >= l) and v_k[l] (k < l).  After the barrier every CTA sums the parts (through
// distributed shared memory) and forms the reflector, w_c = v^H P[:, c] = P[l][c] +
// conj(inv) d_c and g_k = v_k^H v = conj(v_k[l]) + inv h_k.  The parts are double-buffered
// by the parity of l: a CTA rewrites a buffer only after the next barrier, which every
// other CTA passes after its reads.  Task q (0..31) of reflector l is sigma (q = 0), d_{l+q}
// (l + q < 32) or h_{l+q-32}, and its part goes to entry q; warp w forms tasks w and w + 16
// in one pass over the rows.
constexpr int kQp = 1 + 2 * kB;   // parts per CTA: sigma, d_c or h_k (entries 1..31), pivot row / v_k[l] (33..64)
constexpr int kTQ = 512;          // threads of the cluster panel QR
constexpr int kWQ = kTQ / 32;
__global__ void __launch_bounds__(kTQ, 1) panel_qr_cluster_kernel(PanelArgs a) {
    extern __shared__ __align__(16) cdf s_qc[];   // P[l * ch + u], rows rho0 + u; then F[u]
    __shared__ cdf s_wp[2][kQp];                  // this CTA's parts, by parity of l
    __shared__ cdf s_w[kQp];                      // their sums over the cluster (pivot entries from the owner)
    __shared__ cdf s_T[kB][kB + 1];               // rank 0: the T factor
    __shared__ cdf s_G[kB][kB + 1];               // rank 0: g of reflector l (row l), tau_l on its diagonal
    __shared__ cdf s_tau, s_inv;
    __shared__ float2 s_beta;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t rank = cluster_rank();
    const int CQ = gridDim.x;   // the grid is one cluster
    const int ch = (a.m + CQ - 1) / CQ;
    const int rho0 = (int)rank * ch, nown = max(0, min(a.m, rho0 + ch) - rho0);
    const int n = a.n;
    cdf* P = s_qc;
    cdf* F = s_qc + (size_t)kB * ch;   // -conj(tau) v of the own rows
    // rank 0: column j of T, T[0:j, j] = -tau_j T[0:j, 0:j] g_j (warp i: row i)
    auto t_column = [&](int j) {
        const cdf tj = s_G[j][j];
        for (int i = wid; i <= j; i += kWQ) {
            if (i == j) {
                if (lane == 0) s_T[j][j] = tj;
            } else {
                CAcc acc;
                acc.zero();
                if (lane >= i && lane < j) acc.mac(s_T[i][lane], s_G[j][lane]);
                const cdf sum = cacc_warp_sum(acc);
                if (lane == 0) s_T[i][j] = cdf_mul(negc(tj), sum);
            }
        }
    };
    for (int e = tid; e < kB * ch; e += kTQ) {
        const int l = e / ch, u = e - l * ch;
        P[e] = u < nown ? __ldcg(a.A + (size_t)(a.c0 + l) * n + a.r1 + rho0 + u) : cdf_zero();
    }
    __syncthreads();
    // the two columns of task q's products conj(P[ca]) P[cb]
    auto task_cols = [&](int q, int l, int& ca, int& cb) {
        const int cc = l + q;
        if (q == 0) {
            ca = l;
            cb = l;
        } else if (cc < kB) {
            ca = l;
            cb = cc;
        } else {
            ca = cc - kB;
            cb = l;
        }
    };
    for (int l = 0; l < a.nref; ++l) {
        cdf* wp = s_wp[l & 1];
        {
            int ca0, cb0, ca1, cb1;
            task_cols(wid, l, ca0, cb0);
            task_cols(wid + kWQ, l, ca1, cb1);
            CAcc acc0, acc1;
            acc0.zero();
            acc1.zero();
            for (int u = max(0, l + 1 - rho0) + lane; u < nown; u += 32) {
                acc0.dot(P[ca0 * ch + u], P[cb0 * ch + u]);
                acc1.dot(P[ca1 * ch + u], P[cb1 * ch + u]);
            }
            const cdf s0 = cacc_warp_sum(acc0), s1 = cacc_warp_sum(acc1);
            if (lane == 0) {
                wp[wid] = s0;
                wp[wid + kWQ] = s1;
            }
        }
        if (l >= rho0 && l < rho0 + nown && tid < kB) {
            // the pivot row P[l][c] (c >= l) at 1 + kB + (c - l); v_k[l] (k < l) at 1 + kB + (32 - l) + k
            const int u = l - rho0, c = tid;
            if (c >= l)
                wp[1 + kB + (c - l)] = P[c * ch + u];
            else
                wp[1 + kB + (kB - l) + c] = P[c * ch + u];
        }
        cluster_arrive();
        if (rank == 0 && l > 0) t_column(l - 1);   // while the other CTAs finish their parts
        cluster_wait();
        // sums of the parts over the cluster (16 threads per entry, one remote load each),
        // pivot data from the owner
        {
            const int ent = tid >> 4, k = tid & 15;
            cdf x = k < CQ ? ld_cluster_cdf(map_rank(&wp[ent], (uint32_t)k)) : cdf_zero();
            const cdf pv = tid < kB ? ld_cluster_cdf(map_rank(&wp[1 + kB + tid], (uint32_t)(l / ch))) : cdf_zero();
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) x = cdf_add(x, cdf_shfl_xor(x, o));
            if (k == 0) s_w[ent] = x;
            if (tid < kB) s_w[1 + kB + tid] = pv;
        }
        __syncthreads();
        if (tid == 0) {
            cdf tau, inv;
            float2 beta;
            reflector(s_w[1 + kB], make_float2(s_w[0].x, s_w[0].y), tau, inv, beta);
            s_tau = tau;
            s_inv = inv;
            s_beta = beta;
            if (rank == 0) a.tau[l] = tau;
        }
        __syncthreads();
        const cdf tau = s_tau, inv = s_inv, cinv = conjc(inv);
        // w_c and g_k from the sums (kept in the d / h entries: w_c at 1 + (c - l), g_k at 1 + (32 - l) + k)
        if (tid < kB) {
            const int c = tid;
            if (c > l) {
                const cdf d = s_w[c - l];
                s_w[c - l] = cdf_fma(s_w[1 + kB + (c - l)], cinv, d);   // P[l][c] + conj(inv) d_c
            } else if (c < l) {
                const cdf h = s_w[kB - l + c];
                s_w[kB - l + c] = cdf_fma(conjc(s_w[1 + kB + (kB - l) + c]), inv, h);   // conj(v_k[l]) + inv h_k
            }
        }
        // own rows: v in place (beta on the diagonal), F = -conj(tau) v
        const cdf mct = negc(conjc(tau));
        for (int u = tid; u < nown; u += kTQ) {
            const int rho = rho0 + u;
            if (rho < l) continue;
            cdf v;
            if (rho == l) {
                v = onec();
                P[l * ch + u] = make_float4(s_beta.x, s_beta.y, 0.f, 0.f);
            } else {
                v = cdf_mul(P[l * ch + u], inv);
                P[l * ch + u] = v;
            }
            F[u] = cdf_mul(mct, v);
        }
        __syncthreads();
        if (rank == 0 && tid <= l) s_G[l][tid] = tid == l ? tau : s_w[kB - l + tid];   // T column l in the next step
        // P <- P - conj(tau) v w on the own rows >= l, columns > l
        {
            const int u0 = max(0, l - rho0), nr = nown - u0, nc = kB - 1 - l;
            for (int e = tid; e < nc * nr; e += kTQ) {
                const int j = e / nr, u = u0 + e - j * nr, c = l + 1 + j;
                P[c * ch + u] = cdf_fma(P[c * ch + u], F[u], s_w[c - l]);
            }
        }
        __syncthreads();
    }
    // the panel ([R; 0]), the reflectors and T back to global memory (the last column of T first)
    if (rank == 0) {
        if (a.nref > 0) t_column(a.nref - 1);
        __syncthreads();
        for (int e = tid; e < kB * kB; e += kTQ) {
            const int r = e >> 5, c = e & 31;
            a.T[e] = r <= c && c < a.nref ? s_T[r][c] : cdf_zero();
        }
    }
    for (int e = tid; e < kB * ch; e += kTQ) {
        const int l = e / ch, u = e - l * ch;
        if (u >= nown) continue;
        const int rho = rho0 + u;
        const cdf x = P[e];
        const bool below = l < a.nref && rho > l;   // v_l stored in place
        a.A[(size_t)(a.c0 + l) * n + a.r1 + rho] = below ? cdf_zero() : x;
        a.V[(size_t)l * n + a.r1 + rho] = l >= a.nref || rho < l ? cdf_zero() : (rho == l ? onec() : x);
    }
    cluster_sync_all();   // no CTA leaves while another may still read its shared memory
}

// ---------------------------------------------------------------------------
// 32 x 32 Gram products X^H Y over rows r1 .. r1 + m - 1 of two [32][n] arrays:
// part[blk][i][j] = sum over the CTA's rows of conj(X[i][r]) Y[j][r]
// (1024 threads, thread (i, j); rows staged in shared memory 32 at a time).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024, 1) gram32_kernel(const cdf* __restrict__ X, const cdf* __restrict__ Y, int n,
                                                         int r1, int m, cdf* part) {
    __shared__ cdf xs[kB][33], ys[kB][33];
    const int tid = threadIdx.x, i = tid >> 5, j = tid & 31;
    const int q0 = blockIdx.x * kGramRows, q1 = min(m, q0 + kGramRows);
    CAcc acc;
    acc.zero();
    for (int q = q0; q < q1; q += 32) {
        const int cnt = min(32, q1 - q);
        // thread (i, j): row q + j of column i
        xs[i][j] = j < cnt ? __ldcg(X + (size_t)i * n + r1 + q + j) : cdf_zero();
        ys[i][j] = j < cnt ? __ldcg(Y + (size_t)i * n + r1 + q + j) : cdf_zero();
        __syncthreads();
        for (int u = 0; u < cnt; ++u) acc.dot(xs[i][u], ys[j][u]);
        __syncthreads();
    }
    part[(size_t)blockIdx.x * kB * kB + i * kB + j] = acc.get();
}

// Y = Z T (Z summed over the K splits), rows r1 .. n-1, into Y[32][n] (a warp per row,
// lane = column of Y)
__global__ void ysum_kernel(const cdf* __restrict__ zpart, int nks, int m, const cdf* __restrict__ T, int n, int r1,
                            cdf* Y) {
    __shared__ cdf Ts[kB][kB + 1];
    for (int e = threadIdx.x; e < kB * kB; e += blockDim.x) Ts[e >> 5][e & 31] = T[e];
    __syncthreads();
    const int rho = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (rho >= m) return;
    cdf z = cdf_zero();
    for (int k = 0; k < nks; ++k) z = cdf_add(z, zpart[((size_t)k * m + rho) * kB + lane]);
    CAcc acc;
    acc.zero();
    for (int l = 0; l < kB; ++l) {
        const cdf zl = make_float4(__shfl_sync(0xffffffffu, z.x, l), __shfl_sync(0xffffffffu, z.y, l),
                                   __shfl_sync(0xffffffffu, z.z, l), __shfl_sync(0xffffffffu, z.w, l));
        if (l <= lane) acc.mac(zl, Ts[l][lane]);
    }
    Y[(size_t)lane * n + r1 + rho] = acc.get();
}

// M = T^H S with S = V^H Y summed from the parts (1024 threads, thread (i, j))
__global__ void __launch_bounds__(1024, 1) mfactor_kernel(const cdf* __restrict__ spart, int ng,
                                                          const cdf* __restrict__ T, cdf* M) {
    __shared__ cdf S[kB][kB + 1], Ts[kB][kB + 1];
    const int tid = threadIdx.x, i = tid >> 5, j = tid & 31;
    cdf s = cdf_zero();
#pragma unroll 8
    for (int k = 0; k < ng; ++k) s = cdf_add(s, __ldcg(spart + (size_t)k * kB * kB + i * kB + j));
    S[i][j] = s;
    Ts[i][j] = T[i * kB + j];
    __syncthreads();
    CAcc acc;
    acc.zero();
    for (int k = 0; k <= i; ++k) acc.dot(Ts[k][i], S[k][j]);   // conj(T[k][i]) S[k][j]
    M[i * kB + j] = acc.get();
}

// W = Y - 1/2 V M, in place over Y (a warp per row, lane = column)
__global__ void wfinal_kernel(const cdf* __restrict__ V, const cdf* __restrict__ M, int n, int r1, int m, cdf* W) {
    __shared__ cdf Ms[kB][kB + 1];
    for (int e = threadIdx.x; e < kB * kB; e += blockDim.x) Ms[e >> 5][e & 31] = M[e];
    __syncthreads();
    const int rho = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (rho >= m) return;
    const cdf v = __ldcg(V + (size_t)lane * n + r1 + rho);
    CAcc acc;
    acc.zero();
    for (int k = 0; k < kB; ++k) {
        const cdf vk = make_float4(__shfl_sync(0xffffffffu, v.x, k), __shfl_sync(0xffffffffu, v.y, k),
                                   __shfl_sync(0xffffffffu, v.z, k), __shfl_sync(0xffffffffu, v.w, k));
        acc.mac(vk, Ms[k][lane]);
    }
    cdf* w = W + (size_t)lane * n + r1 + rho;
    *w = cdf_fma(*w, make_float4(-0.5f, 0.f, 0.f, 0.f), acc.get());
}

// ---------------------------------------------------------------------------
// Stage 2: bulge chasing (cooperative; sweeps i = blockIdx.x, blockIdx.x + G, ...).
// Task t of sweep i has the window rows and columns [p, q), p = i + 1 + 32 t,
// q = min(p + 32, n); it reflects column cc = (t == 0 ? i : p - 32) on rows
// [p, q) (rows below p zeroed), applies the reflector to the block left of the
// window ([p, q) x [p - 32, p), t >= 1, kept in shared memory from task t - 1),
// to the window's diagonal block (both sides) and to the block below
// ([q, q + 32) x [p, q), right), which becomes the next task's left block.
// Shared memory: three 32 x 33 blocks (D, and the left and below blocks, whose
// roles swap from task to task) and five vectors.
// ---------------------------------------------------------------------------
struct BulgeArgs {
    cdf* A;
    int n;
    int* prog;   // [n] crit count of each sweep (kSweepDone once it has ended), zero on entry
    int* pre;    // [n] pre count of each sweep (kSweepDone once it has ended), zero on entry
    int* err;
    long spin;
};

constexpr int kBlk = kB * (kB + 1);
constexpr size_t kBulgeSmem = sizeof(cdf) * (3 * kBlk + 5 * kB);

// publish a count: every thread's earlier writes were ordered before this by __syncthreads,
// and the release makes them visible before the count (as in the grid barrier)
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ cdf shfl_cdf(cdf v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}
constexpr int kBT = 512;                // threads of the bulge-chasing kernel
constexpr int kBW = kBT / 32;           // its warps

// Each sweep publishes two counts.  crit[i] = t + 2 once the critical part of task t is
// out: column 0 of its window's block after the two-sided update (whose entries, with the
// reflected column's beta, are the only ones the next sweep's task t - 1 still waits for)
// and the reflector of task t + 1.  pre[i] = t once the rest of task t - 1 (the other
// columns of its diagonal block, its block below) and the left-block part of task t are
// out.  Task t of sweep i:
//   deferred part of task t - 1 and left block of task t (no other sweep touches either
//     meanwhile), one column c >= 1 per warp at a time, lane r = row r: D -= v w^H + w v^H
//     written back; the block below of task t - 1 (in shared memory), now the left block L,
//     -= tau z v^H in registers; s_c = (v^H L)_c by one warp sum; L -= conj(tau) v s^H
//     written back; then pre[i] = t;
//   once pre[i-1] >= t + 1 (sweep i - 1 is done with all of the window but its column 31):
//     the window's block (lower triangle) and the block below are loaded but for column
//     31; threads 0..255 form y = D v, threads 256..511 z = B v without those entries (8
//     threads per row, 4 columns each);
//   once crit[i-1] >= t + 3: warp 0 loads D(31,31), completes y, forms mu = v^H y,
//     w = tau y - |tau|^2 mu / 2 v and column 0 of the updated block; warp 1 loads column
//     31 of the block below, completes z and forms R_{t+1} from column 0 of the updated
//     block below, B[:,0] - tau z (v_0 = 1); crit[i] = t + 2.
// The last task of a sweep does all of its work after crit[i-1] >= t + 3.
__global__ void __launch_bounds__(kBT, 1) bulge_kernel(BulgeArgs a) {
    extern __shared__ __align__(16) cdf s_bg[];
    __shared__ int s_ok;
    __shared__ cdf s_tau;
    cdf* D = s_bg;                     // D[r * 33 + c], lower triangle (r >= c)
    cdf* Lb = s_bg + kBlk;             // left block: Lb[r * 33 + c], rows p + r, columns p - 32 + c
    cdf* Bb = s_bg + 2 * kBlk;         // block below: Bb[r * 33 + c], rows q + r, columns p + c
    cdf* vo = s_bg + 3 * kBlk;         // v of the previous task (its deferred part)
    cdf* vs = vo + kB;                 // v of the task
    cdf* vn = vs + kB;                 // v of the next task
    cdf* ys = vn + kB;                 // y, then w
    cdf* zs = ys + kB;                 // z, then tau z
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int half = tid >> 8, r2 = (tid & 255) >> 3, k2 = tid & 7;   // product thread: y or z, row r2
    const int n = a.n;
    cdf* A = a.A;
    auto at = [&](int r, int c) -> cdf* { return A + (size_t)c * n + r; };
    constexpr int S = kB + 1;
    // tid 0 waits until sweep i - 1 has raised count cnt to `need`; false if the wait gave up
    auto wait_prev = [&](const int* cnt, int i, int need) {
        if (tid == 0) {
            bool ok = true;
            if (i > 0) {
                ok = false;
                for (long it = 0; it < a.spin; ++it) {
                    if (ld_acquire_gpu((const unsigned*)(cnt + i - 1)) >= (unsigned)need) {
                        ok = true;
                        break;
                    }
                    if ((it & 255) == 255 && *(volatile int*)a.err) break;
                }
                if (!ok) atomicExch(a.err, 1);
            }
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        return s_ok != 0;
    };
    // the reflector of column x (lane l holds x_l, l < len), in the calling warp
    auto form = [&](cdf xl, int len, cdf& vl, cdf& tau, float2& beta) {
        float sg = 0.f, lo = 0.f;
        if (lane >= 1 && lane < len) {
            df_acc(sg, lo, xl.x, xl.y, xl.x, xl.y);
            df_acc(sg, lo, xl.z, xl.w, xl.z, xl.w);
        }
        const float2 sigma = warp_sum_df(df_fin(sg, lo));
        cdf inv;
        reflector(shfl_cdf(xl, 0), sigma, tau, inv, beta);
        vl = lane == 0 ? onec() : (lane < len ? cdf_mul(xl, inv) : cdf_zero());
    };
    // w = tau y - |tau|^2 mu / 2 v with mu = Re v^H y, in warp 0 (lane l holds y_l, v_l)
    auto form_w = [&](cdf yy, cdf vl, cdf tau, int len) {
        float m0 = 0.f, m1 = 0.f;
        if (lane < len) {
            df_acc(m0, m1, vl.x, vl.y, yy.x, yy.y);
            df_acc(m0, m1, vl.z, vl.w, yy.z, yy.w);
        }
        const float2 mu = warp_sum_df(df_fin(m0, m1));
        float t0 = 0.f, t1 = 0.f;
        df_acc(t0, t1, tau.x, tau.y, tau.x, tau.y);
        df_acc(t0, t1, tau.z, tau.w, tau.z, tau.w);
        const float2 cf = df_mul(df_mul(df_fin(t0, t1), mu), make_float2(-0.5f, 0.f));
        return lane < len ? cdf_fma(cdf_mul(tau, yy), make_float4(cf.x, cf.y, 0.f, 0.f), vl) : cdf_zero();
    };
    for (int i = blockIdx.x; i < n - 2; i += gridDim.x) {
        cdf vl, tau;   // lane l of every warp holds v_l
        float2 beta;
        // R_0: column i on rows i+1 .. i+32, final once sweep i - 1 has done the critical part of task 0
        {
            const int p = i + 1, len = min(p + kB, n) - p;
            if (!wait_prev(a.prog, i, 2)) return;
            const cdf xl = lane < len ? __ldcg(at(p + lane, i)) : cdf_zero();
            form(xl, len, vl, tau, beta);
            if (wid == 0) {
                vs[lane] = vl;
                if (lane < len) *at(p + lane, i) = lane == 0 ? make_float4(beta.x, beta.y, 0.f, 0.f) : cdf_zero();
            }
            __syncthreads();
            if (tid == 0) st_release_gpu(a.prog + i, 1);
        }
        for (int t = 0;; ++t) {
            const int p = i + 1 + kB * t;
            const int q = min(p + kB, n), len = q - p;
            const int qb = min(q + kB, n), lenb = qb - q;
            const bool next = q <= n - 2;   // a task follows; then len == 32
            if (t > 0) {
                // deferred part of task t - 1 (whose window [p - 32, p) is full) and the left
                // block of task t, column by column: warp w takes columns w and w + 16, lane r
                // row r; the block below of task t - 1 is updated in registers, s_c formed by
                // one warp sum and the left block's update written back
                const int pp = p - kB;
                const cdf f = cdf_mul(negc(conjc(tau)), vl);   // -conj(tau) v_r of this task
                const cdf zr = zs[lane], vor = vo[lane], wr = ys[lane];   // task t - 1: tau z_r, v_r, w_r
                for (int c = wid + (wid == 0 ? kBW : 0); c < kB; c += kBW) {   // column 0 needs neither
                    if (lane >= c) *at(pp + lane, pp + c) = cdf_rank2(D[lane * S + c], vor, wr, ys[c], vo[c]);
                    const cdf x = lane < len ? cdf_fma(Lb[lane * S + c], negc(zr), conjc(vo[c])) : cdf_zero();
                    CAcc as;
                    as.zero();
                    as.dot(vl, x);
                    const cdf sc = cacc_warp_sum(as);
                    if (lane < len) *at(p + lane, p - kB + c) = cdf_fma(x, f, sc);
                }
                __syncthreads();
                if (tid == 0) st_release_gpu(a.pre + i, t);
            }
            if (!(next ? wait_prev(a.pre, i, t + 1) : wait_prev(a.prog, i, t + 3))) return;
            for (int e = tid; e < kB * kB; e += kBT) {
                const int r = e & 31, c = e >> 5;
                const bool late = next && c == kB - 1;   // column 31: after crit[i-1] >= t + 3
                if (r >= c && r < len && !late) D[r * S + c] = __ldcg(at(p + r, p + c));
                if (r < lenb && c < len && !late) Bb[r * S + c] = __ldcg(at(q + r, p + c));
            }
            __syncthreads();
            {   // y = D v (threads 0..255), z = B v (threads 256..511), without column 31 when a task follows
                CAcc acc;
                acc.zero();
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = 4 * k2 + u;
                    const cdf vc = shfl_cdf(vl, c);
                    if (half == 0) {
                        if (r2 < len && c < len && !(next && r2 == kB - 1 && c == kB - 1))
                            acc.mac(r2 >= c ? D[r2 * S + c] : conjc(D[c * S + r2]), vc);
                    } else {
                        if (r2 < lenb && c < len && !(next && c == kB - 1)) acc.mac(Bb[r2 * S + c], vc);
                    }
                }
                const cdf rs = cacc_group_sum<8>(acc);
                if (k2 == 0) {
                    if (half == 0)
                        ys[r2] = rs;
                    else
                        zs[r2] = rs;
                }
            }
            if (!next) {   // the last task: w, tau z, then every update
                __syncthreads();
                if (wid == 0)
                    ys[lane] = form_w(ys[lane], vl, tau, len);
                else if (wid == 1)
                    zs[lane] = cdf_mul(tau, zs[lane]);
                __syncthreads();
                for (int e = tid; e < kB * kB; e += kBT) {
                    const int r = e & 31, c = e >> 5;
                    if (c <= r && r < len) *at(p + r, p + c) = cdf_rank2(D[r * S + c], vs[r], ys[r], ys[c], vs[c]);
                    if (r < lenb && c < len) *at(q + r, p + c) = cdf_fma(Bb[r * S + c], negc(zs[r]), conjc(vs[c]));
                }
                __syncthreads();
                if (tid == 0) {
                    st_release_gpu(a.pre + i, kSweepDone);
                    st_release_gpu(a.prog + i, kSweepDone);
                }
                break;
            }
            if (!wait_prev(a.prog, i, t + 3)) return;   // its barrier also orders the partial sums
            if (wid == 0) {   // D(31,31), y, w, column 0 of the updated block
                cdf yy = ys[lane];
                const cdf v31 = shfl_cdf(vl, kB - 1);
                if (lane == kB - 1) {
                    const cdf d = __ldcg(at(p + kB - 1, p + kB - 1));
                    D[(kB - 1) * S + kB - 1] = d;
                    yy = cdf_fma(yy, d, v31);
                }
                const cdf w = form_w(yy, vl, tau, kB);
                ys[lane] = w;
                *at(p + lane, p) = cdf_rank2(D[lane * S], vl, w, shfl_cdf(w, 0), shfl_cdf(vl, 0));
            } else if (wid == 1) {   // column 31 of the block below, tau z, R_{t+1}
                const cdf v31 = shfl_cdf(vl, kB - 1);
                cdf zz = zs[lane], b0 = cdf_zero();
                if (lane < lenb) {
                    const cdf b = __ldcg(at(q + lane, p + kB - 1));
                    Bb[lane * S + kB - 1] = b;
                    zz = cdf_fma(zz, b, v31);
                    b0 = Bb[lane * S];
                }
                const cdf tz = cdf_mul(tau, zz);
                zs[lane] = tz;
                const cdf xl = lane < lenb ? cdf_fma(b0, negc(tz), onec()) : cdf_zero();
                cdf vln, taun;
                float2 betan;
                form(xl, lenb, vln, taun, betan);
                vn[lane] = vln;
                if (lane == 0) s_tau = taun;
                const cdf xo = lane == 0 ? make_float4(betan.x, betan.y, 0.f, 0.f) : cdf_zero();
                Bb[lane * S] = xo;
                if (lane < lenb) *at(q + lane, p) = xo;
            }
            __syncthreads();
            if (tid == 0) st_release_gpu(a.prog + i, t + 2);
            vl = vn[lane];
            tau = s_tau;
            cdf* tv = vo;   // v of this task stays for its deferred part
            vo = vs;
            vs = vn;
            vn = tv;
            cdf* tb = Lb;   // the block below becomes the next task's left block
            Lb = Bb;
            Bb = tb;
        }
        __syncthreads();
    }
}

// d_i = Re A[i,i], e_i = |A[i+1,i]| (FP64)
__global__ void band_extract_kernel(const cdf* __restrict__ A, int n, double* d, double* e) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cdf a = __ldcg(A + (size_t)i * n + i);
    d[i] = (double)a.x + (double)a.y;
    if (i + 1 < n) {
        const cdf b = __ldcg(A + (size_t)i * n + i + 1);
        const double re = (double)b.x + (double)b.y, im = (double)b.z + (double)b.w;
        e[i] = sqrt(re * re + im * im);
    } else {
        e[i] = 0.0;
    }
}

}  // namespace

size_t tridiag2_bytes(int64_t n) {
    const int64_t ng = (n + kGramRows - 1) / kGramRows;
    // H0 vectors (3 n); A22 V parts (kMaxKs n 32); Gram parts (ng 1024); T, M (2 x 1024); tau, pivots
    // (64); partial norms (256 float2); partial w and g (256 x 64); progress (2 n ints); barrier; alignment
    return sizeof(cdf) * (size_t)(3 * n + kMaxKs * n * kB + ng * kB * kB + 2 * kB * kB + 2 * kB + 512 * kB) +
           sizeof(float2) * 256 + 2 * sizeof(int) * (size_t)n + zgemm_tc_bytes(n) + 64 + 16 * 256;
}

int launch_tridiag2(cdf* A, int64_t n64, const double2* v0, const double* beta0, double* d, double* e, cdf* V, cdf* W,
                    void* tc_scratch, void* scratch, int* err, cudaStream_t st, long wait_polls) {
    const int n = (int)n64;
    char* p = (char*)scratch;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)q;
    };
    const int64_t ngmax = (n + kGramRows - 1) / kGramRows;
    cdf* hy = (cdf*)take(sizeof(cdf) * n);
    cdf* hv = (cdf*)take(sizeof(cdf) * n);
    cdf* hw = (cdf*)take(sizeof(cdf) * n);
    cdf* zpart = (cdf*)take(sizeof(cdf) * (size_t)kMaxKs * n * kB);
    cdf* spart = (cdf*)take(sizeof(cdf) * (size_t)ngmax * kB * kB);
    cdf* T = (cdf*)take(sizeof(cdf) * kB * kB);
    cdf* M = (cdf*)take(sizeof(cdf) * kB * kB);
    cdf* tau = (cdf*)take(sizeof(cdf) * kB);
    cdf* piv = (cdf*)take(sizeof(cdf) * kB);
    float2* part = (float2*)take(sizeof(float2) * 256);
    cdf* wpart = (cdf*)take(sizeof(cdf) * 256 * 2 * kB);
    int* prog = (int*)take(sizeof(int) * n);
    int* pre = (int*)take(sizeof(int) * n);
    unsigned* bar = (unsigned*)take(sizeof(unsigned));
    void* zscratch = take(zgemm_tc_bytes(n));
    const long spin = wait_limit(wait_polls, kGridSpinLimit);

    int dev = 0, sms = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t nn = (int64_t)n * n;
    to_cdf_kernel<<<sms * 4, kT2, 0, st>>>(A, nn);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    // start reflector
    h0_matvec_kernel<<<(unsigned)((n + kW2 - 1) / kW2), kT2, 0, st>>>(A, n, v0, hy);
    note_launch();
    h0_vectors_kernel<<<1, kT2, 0, st>>>(v0, beta0, hy, n, hv, hw);
    note_launch();
    rank2_all_kernel<<<sms * 4, kT2, 0, st>>>(A, n, hv, hw);
    note_launch();
    BSE_CUDA(cudaGetLastError());

    // the panel QR on one cluster of CQ CTAs (16, else 8) when the rows of the largest panel
    // fit its shared memory, else on co-resident CTAs with grid barriers
    int CQ = 0;
    {
        const int m0 = n - kB;
        for (int cq : {16, 8}) {
            if (m0 < 2) break;
            const int ch = (m0 + cq - 1) / cq;
            const size_t smem = sizeof(cdf) * (kB + 1) * (size_t)ch;
            if (smem > 200 * 1024) continue;
            if (cq > 8 &&
                cudaFuncSetAttribute(panel_qr_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                    cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (cudaFuncSetAttribute(panel_qr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = cq;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(cq);
            cfg.blockDim = dim3(kTQ);
            cfg.dynamicSmemBytes = smem;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, (void*)panel_qr_cluster_kernel, &cfg) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (nc >= 1) {
                CQ = cq;
                break;
            }
        }
    }

    // stage 1: panels of 32 columns
    for (int c0 = 0;; c0 += kB) {
        const int r1 = c0 + kB, m = n - r1;
        if (m < 2) break;
        const int nref = std::min(kB, m - 1);
        // panel QR on Gq co-resident CTAs of one row each per thread
        int Gq = std::max((m + 159) / 160, std::min(kQrMaxCta, (m + 31) / 32));
        Gq = std::min(Gq, sms);
        const int ch = (m + Gq - 1) / Gq;
        const size_t qsm = sizeof(cdf) * 2 * kB * (size_t)ch;
        if (ch > kT2) return fail(BSE_EUNSUPPORTED, "two-stage reduction: n = %d too large for the panel QR", n);
        BSE_CUDA(cudaFuncSetAttribute(panel_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm));
        BSE_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
        PanelArgs pa;
        pa.A = A;
        pa.n = n;
        pa.c0 = c0;
        pa.r1 = r1;
        pa.m = m;
        pa.nref = nref;
        pa.V = V;
        pa.tau = tau;
        pa.part = part;
        pa.piv = piv;
        pa.wpart = wpart;
        pa.T = T;
        pa.bar = bar;
        pa.err = err;
        pa.spin = spin;
        if (CQ > 0) {
            const int chq = (m + CQ - 1) / CQ;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = CQ;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(CQ);
            cfg.blockDim = dim3(kTQ);
            cfg.dynamicSmemBytes = sizeof(cdf) * (kB + 1) * (size_t)chq;
            cfg.stream = st;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            BSE_CUDA(cudaLaunchKernelEx(&cfg, panel_qr_cluster_kernel, pa));
        } else {
            void* qargs[] = {&pa};
            BSE_CUDA(cudaLaunchCooperativeKernel((const void*)panel_qr_kernel, dim3(Gq), dim3(kT2), qargs, qsm, st));
        }
        note_launch();
        const int ng = (m + kGramRows - 1) / kGramRows;
        // Z = A22 V split over K, Y = Z T
        const int ks = zgemm_tc_splits(m, sms);
        BSE_TRY(launch_zgemm_tc(A, n, r1, m, V, zscratch, zpart, ks, err, st, wait_polls));
        ysum_kernel<<<(unsigned)((m + kW2 - 1) / kW2), kT2, 0, st>>>(zpart, ks, m, T, n, r1, W);
        note_launch();
        // W = Y - 1/2 V T^H V^H Y
        gram32_kernel<<<ng, 1024, 0, st>>>(V, W, n, r1, m, spart);
        note_launch();
        mfactor_kernel<<<1, 1024, 0, st>>>(spart, ng, T, M);
        note_launch();
        wfinal_kernel<<<(unsigned)((m + kW2 - 1) / kW2), kT2, 0, st>>>(V, M, n, r1, m, W);
        note_launch();
        BSE_CUDA(cudaGetLastError());
        // A22 -= V W^H + W V^H on the tensor cores
        BSE_TRY(launch_panel_update_tc(A, n, r1, 0, V, W, tc_scratch, err, st, wait_polls));
    }

    // stage 2: bulge chasing
    if (n > 2) {
        BSE_CUDA(cudaMemsetAsync(prog, 0, sizeof(int) * n, st));
        BSE_CUDA(cudaMemsetAsync(pre, 0, sizeof(int) * n, st));
        BSE_CUDA(cudaFuncSetAttribute(bulge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBulgeSmem));
        int per_sm = 0;
        BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bulge_kernel, kBT, kBulgeSmem));
        if (per_sm < 1) return fail(BSE_EUNSUPPORTED, "bulge-chasing kernel cannot be resident");
        const int G = std::min(sms, n - 2);
        BulgeArgs ba;
        ba.A = A;
        ba.n = n;
        ba.prog = prog;
        ba.pre = pre;
        ba.err = err;
        ba.spin = spin;
        void* bargs[] = {&ba};
        BSE_CUDA(cudaLaunchCooperativeKernel((const void*)bulge_kernel, dim3(G), dim3(kBT), bargs, kBulgeSmem, st));
        note_launch();
    }
    band_extract_kernel<<<(unsigned)((n + kT2 - 1) / kT2), kT2, 0, st>>>(A, n, d, e);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

}  // namespace bse
