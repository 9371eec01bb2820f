// FP64 CUDA kernels of the symmetry-reduced BSE block builder (sm_103a).
//
// Paper references: Eq. w_interaction (pair densities in plane waves),
// Eq. BSE-eigval (H = D + spin K^x - K^d), Eq. Wdiv with divergence_int and
// divergence_sum (head correction), Eq. Ts (band rotations), Eqs. projection
// and transformationU (projection onto an irrep), Eqs. oscillator,
// oscillatorA, reducible_polar (spectrum).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>

#include "dfloat.h"
#include "fp64_fast.h"
#include "internal.h"

namespace bse {

// process-wide count of kernel launches made by this library
static std::atomic<long long> g_launches{0};
int64_t launches_total() { return g_launches.load(); }
void note_launch() { g_launches.fetch_add(1); }

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc += conj(a) * b
__device__ __forceinline__ void cfma_conj(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

#define LAUNCH_CHECK()                                                                  \
    do {                                                                                \
        g_launches.fetch_add(1);                                                        \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess)                                                          \
            return fail(BSE_ECUDA, "%s:%d launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------
// mesh helpers
// ---------------------------------------------------------------------------
// q = k - k' on the mesh and the integer fold f_k' + f_q - f_k
__device__ __forceinline__ int mesh_minus(const DevSys& S, int k, int kp, int fold[3]) {
    const int n[3] = {S.n1, S.n2, S.n3};
    int iq[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int ik = S.kidx[3 * k + a], ikp = S.kidx[3 * kp + a];
        iq[a] = (ik - ikp + n[a]) % n[a];
        fold[a] = (ikp + iq[a] - ik) / n[a];
    }
    return (iq[0] * S.n2 + iq[1]) * S.n3 + iq[2];
}

// position of integer vector m in the coset sphere of k, -1 if absent
__device__ __forceinline__ int sphere_index(const DevSys& S, int k, int m0, int m1, int m2) {
    int x0 = m0 - S.blo[0], x1 = m1 - S.blo[1], x2 = m2 - S.blo[2];
    if ((unsigned)x0 >= (unsigned)S.bdim[0] || (unsigned)x1 >= (unsigned)S.bdim[1] ||
        (unsigned)x2 >= (unsigned)S.bdim[2])
        return -1;
    return S.box[(int64_t)k * S.bvol + ((int64_t)x0 * S.bdim[1] + x1) * S.bdim[2] + x2];
}

// ---------------------------------------------------------------------------
// band rotations (Eq. Ts): map p -> R^{-T} p and its phase exp(-2 pi i R^{-T}p . t)
// ---------------------------------------------------------------------------
__global__ void rotmap_kernel(DevSys S, const int* __restrict__ rk, const double* __restrict__ tau,
                              const int* __restrict__ rotk, int nops, int* perm, double2* phase) {
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = (int64_t)nops * S.nk * S.npw_max;
    if (id >= tot) return;
    int i = (int)(id % S.npw_max);
    int k = (int)((id / S.npw_max) % S.nk);
    int s = (int)(id / ((int64_t)S.npw_max * S.nk));
    if (i >= S.npw[k]) {
        perm[id] = -1;
        phase[id] = make_double2(0.0, 0.0);
        return;
    }
    const int* R = rk + 9 * s;
    const int k2 = rotk[(int64_t)s * S.nk + k];
    // 1/n by a Newton reciprocal (an FP64 divide costs hundreds of cycles of
    // GB300's FP64 pipe); fr - f2 is an integer up to rounding, f2 enters the phase
    const double rn[3] = {rcp_nr((double)S.n1), rcp_nr((double)S.n2), rcp_nr((double)S.n3)};
    const int* m = S.gk + ((int64_t)k * S.npw_max + i) * 3;
    int mr[3];
    double th = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double fr = 0.0;
        int mm = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            fr += R[3 * a + b] * (S.kidx[3 * k + b] * rn[b]);
            mm += R[3 * a + b] * m[b];
        }
        double f2 = S.kidx[3 * k2 + a] * rn[a];
        int fold = (int)rint(fr - f2);
        mr[a] = mm + fold;
        th += (f2 + mr[a]) * tau[3 * s + a];
    }
    th -= floor(th);
    double sn, cs;
    sincospi(-2.0 * th, &sn, &cs);
    perm[id] = sphere_index(S, k2, mr[0], mr[1], mr[2]);
    phase[id] = make_double2(cs, sn);
}

// Gamma(s)_{k n}^{sk n'} = sum_p conj(c_{sk n'}(R^{-T} p)) exp(..) c_{k n}(p)
__global__ void gamma_kernel(DevSys S, int nops, const int* __restrict__ rotk, const int* __restrict__ perm,
                             const double2* __restrict__ phase, const int* __restrict__ ent, int64_t n_ent,
                             double2* out) {
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)nops * n_ent) return;
    int64_t e = id % n_ent;
    int s = (int)(id / n_ent);
    int k = ent[3 * e], np_ = ent[3 * e + 1], nb_ = ent[3 * e + 2];
    int k2 = rotk[(int64_t)s * S.nk + k];
    const double2* ck = S.coef + ((int64_t)k * S.nb + nb_) * S.npw_max;
    const double2* ck2 = S.coef + ((int64_t)k2 * S.nb + np_) * S.npw_max;
    const int64_t base = ((int64_t)s * S.nk + k) * S.npw_max;
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < S.npw[k]; ++i) {
        int j = perm[base + i];
        if (j < 0) continue;
        cfma_conj(acc, ck2[j], cmul(phase[base + i], ck[i]));
    }
    out[id] = acc;
}

int launch_rotmap(const DevSys& s, const int* rk, const double* tau, const int* rotk, int nops, int* perm,
                  double2* phase, cudaStream_t st) {
    int64_t n = (int64_t)nops * s.nk * s.npw_max;
    rotmap_kernel<<<ceil_div(n, 256), 256, 0, st>>>(s, rk, tau, rotk, nops, perm, phase);
    LAUNCH_CHECK();
    return BSE_OK;
}

int launch_gamma(const DevSys& s, int nops, const int* rotk, const int* perm, const double2* phase, const int* ent,
                 int64_t n_ent, double2* out, cudaStream_t st) {
    int64_t n = (int64_t)nops * n_ent;
    if (n == 0) return BSE_OK;
    gamma_kernel<<<ceil_div(n, 128), 128, 0, st>>>(s, nops, rotk, perm, phase, ent, n_ent, out);
    LAUNCH_CHECK();
    return BSE_OK;
}

// ---------------------------------------------------------------------------
// pair densities (Eq. w_interaction in plane waves)
// ---------------------------------------------------------------------------
// shared-memory staging of one k pair: coefficients of both k and the
// index table idx[g][j] = position of p'_j + Q_g in S_k (or -1).  V is the
// complex type of the coefficients (double2, or float2 for the FP32 copy the
// mixed builds compute their pair densities from).
template <typename V>
struct PairStage {
    V* ck;          // [nb][npw_max]
    V* ckp;         // [nb][npw_max]
    short* idx;     // [ng][npkp]
    int q, ng, npkp;
};

template <typename V>
__device__ void stage_pair(const DevSys& S, const V* __restrict__ coef, int k, int kp, PairStage<V>& P) {
    int fold[3];
    P.q = mesh_minus(S, k, kp, fold);
    P.ng = S.ng[P.q];
    P.npkp = S.npw[kp];
    const int tot = S.nb * S.npw_max;
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        P.ck[e] = coef[(int64_t)k * tot + e];
        P.ckp[e] = coef[(int64_t)kp * tot + e];
    }
    const int* gq = S.gq + (int64_t)P.q * S.ng_max * 3;
    const int* gk = S.gk + (int64_t)kp * S.npw_max * 3;
    for (int e = threadIdx.x; e < P.ng * P.npkp; e += blockDim.x) {
        int g = e / P.npkp, j = e % P.npkp;
        P.idx[e] = (short)sphere_index(S, k, gk[3 * j] + gq[3 * g] + fold[0], gk[3 * j + 1] + gq[3 * g + 1] + fold[1],
                                       gk[3 * j + 2] + gq[3 * g + 2] + fold[2]);
    }
}

__device__ __forceinline__ void cfma_conj_any(double2& acc, double2 a, double2 b) { cfma_conj(acc, a, b); }
__device__ __forceinline__ void cfma_conj_any(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

// rho[a][b][g] for bands n = n_lo + a (a < nn), n' = np_lo + b (b < nnp), in the precision of V
template <typename V>
__device__ __forceinline__ V rho_elem(const DevSys& S, const PairStage<V>& P, int n, int np_, int g) {
    const V* cn = P.ck + n * S.npw_max;
    const V* cp = P.ckp + np_ * S.npw_max;
    const short* row = P.idx + g * P.npkp;
    V acc;
    acc.x = 0;
    acc.y = 0;
    for (int j = 0; j < P.npkp; ++j) {
        int i = row[j];
        if (i >= 0) cfma_conj_any(acc, cn[i], cp[j]);
    }
    return acc;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t stage_bytes(int cplx_bytes, int nb, int npw_max, int ng_max) {
    return align16((size_t)cplx_bytes * nb * npw_max) * 2 + align16(sizeof(short) * (size_t)ng_max * npw_max);
}

template <typename V>
__global__ void pairdens_kernel(DevSys S, const V* __restrict__ coef, const int* __restrict__ kk,
                                const int* __restrict__ kpp, int bands, int exchange_layout, V* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    PairStage<V> P;
    const size_t cb = align16(sizeof(V) * (size_t)S.nb * S.npw_max);
    P.ck = (V*)smem;
    P.ckp = (V*)(smem + cb);
    P.idx = (short*)(smem + 2 * cb);
    const int64_t pr = blockIdx.x;
    const int k = kk[pr], kp = kpp[pr];
    stage_pair(S, coef, k, kp, P);
    __syncthreads();
    int n_lo, nn, np_lo, nnp;
    if (bands == BSE_BANDS_CC) { n_lo = S.nv; nn = S.nc; np_lo = S.nv; nnp = S.nc; }
    else if (bands == BSE_BANDS_VV) { n_lo = 0; nn = S.nv; np_lo = 0; nnp = S.nv; }
    else { n_lo = S.nv; nn = S.nc; np_lo = 0; nnp = S.nv; }
    if (!exchange_layout) {
        const int tot = nn * nnp * S.ng_max;
        V* o = out + pr * (int64_t)tot;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            int g = e % S.ng_max, ab = e / S.ng_max;
            V z;
            z.x = 0;
            z.y = 0;
            o[e] = g < P.ng ? rho_elem(S, P, n_lo + ab / nnp, np_lo + ab % nnp, g) : z;
        }
    } else {
        // exchange vectors P[(k*nv + v)*nc + c][g] = m^k_cv(G_g), q = 0
        const int ng0 = P.ng;
        const int tot = nn * nnp * ng0;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            int g = e % ng0, ab = e / ng0;
            int c = ab / nnp, v = ab % nnp;
            out[(((int64_t)k * S.nv + v) * S.nc + c) * ng0 + g] = rho_elem(S, P, n_lo + c, np_lo + v, g);
        }
    }
}

template <typename V>
static int launch_pairdens_t(const DevSys& s, const V* coef, const int* k, const int* kp, int64_t npairs, int bands,
                             int exchange_layout, V* out, cudaStream_t st) {
    if (npairs == 0) return BSE_OK;
    size_t sm = stage_bytes((int)sizeof(V), s.nb, s.npw_max, s.ng_max);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(pairdens_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return fail(BSE_ECUDA, "pairdens smem %zu: %s", sm, cudaGetErrorString(e));
    }
    pairdens_kernel<V><<<(unsigned)npairs, 256, sm, st>>>(s, coef, k, kp, bands, exchange_layout, out);
    LAUNCH_CHECK();
    return BSE_OK;
}

int launch_pairdens(const DevSys& s, const int* k, const int* kp, int64_t npairs, int bands, int exchange_layout,
                    double2* out, cudaStream_t st) {
    return launch_pairdens_t(s, s.coef, k, kp, npairs, bands, exchange_layout, out, st);
}

int launch_pairdens32(const DevSys& s, const float2* coef32, const int* k, const int* kp, int64_t npairs, int bands,
                      float2* out, cudaStream_t st) {
    return launch_pairdens_t(s, coef32, k, kp, npairs, bands, 0, out, st);
}

// ---------------------------------------------------------------------------
// projection (Eqs. projection, transformationU), orbit-sparse, two stages:
//   Y = X U_b   (tile rows of star a, columns of star b's basis vectors)
//   H_mu[cols a, cols b] = U_a^dagger Y (+ exchange, projected)
// ---------------------------------------------------------------------------
// FP64 tiles (the FP64 build): FP64 products and sums
template <typename VX>
__global__ void project_right_kernel(DevBasis Bs, const TileTask* __restrict__ tiles, const VX* __restrict__ X,
                                     double2* Y) {
    const TileTask t = tiles[blockIdx.z];
    const int r = blockIdx.x * 32 + threadIdx.x;
    const int64_t ncol = t.cb1 - t.cb0;
    if (r >= t.rows) return;
    const VX* Xt = X + t.xoff;
    for (int64_t jj = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; jj < ncol; jj += (int64_t)gridDim.y * blockDim.y) {
        const int64_t j = t.cb0 + jj;
        const int o = Bs.col_orbit[j];
        const int64_t m0 = Bs.orbit_off[o], n_o = Bs.orbit_off[o + 1] - m0;
        const double2* u = Bs.coef + Bs.col_off[j];
        double2 acc = make_double2(0.0, 0.0);
        for (int64_t tt = 0; tt < n_o; ++tt) {
            VX x = Xt[(int64_t)Bs.member_loc[m0 + tt] * t.rows + r];
            cfma(acc, make_double2((double)x.x, (double)x.y), u[tt]);
        }
        Y[t.yoff + jj * t.rows + r] = acc;
    }
}

// FP32 tiles (the mixed builds): each product of an FP32 element of X with a
// coefficient of U is formed exactly in double-float (TwoProduct) and summed
// in double-float on the FP32 pipe, whose rate is 64 times the FP64 pipe's;
// the sum's error (about 2^-47 relative) is far below that of the FP32 tile
// Y in FP64 (double2) or, for a double-float left projection, in double-float (float4)
__device__ __forceinline__ void store_y(double2* y, float sr, float lr, float si, float li) {
    *y = make_double2((double)sr + (double)lr, (double)si + (double)li);
}
__device__ __forceinline__ void store_y(float4* y, float sr, float lr, float si, float li) {
    *y = make_float4(sr, lr, si, li);
}
template <typename YT>
__global__ void project_right_df_kernel(DevBasis Bs, const TileTask* __restrict__ tiles, const float2* __restrict__ X,
                                        YT* Y) {
    const TileTask t = tiles[blockIdx.z];
    const int r = blockIdx.x * 32 + threadIdx.x;
    const int64_t ncol = t.cb1 - t.cb0;
    if (r >= t.rows) return;
    const float2* Xt = X + t.xoff;
    for (int64_t jj = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; jj < ncol; jj += (int64_t)gridDim.y * blockDim.y) {
        const int64_t j = t.cb0 + jj;
        const int o = Bs.col_orbit[j];
        const int64_t m0 = Bs.orbit_off[o], n_o = Bs.orbit_off[o + 1] - m0;
        const float4* u = Bs.coef_df + Bs.col_off[j];
        // raw double-float sums (leading words by TwoSum, every error and low part in the
        // low words), normalised once at the end
        float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
#pragma unroll 4
        for (int64_t tt = 0; tt < n_o; ++tt) {
            const float2 x = Xt[(int64_t)Bs.member_loc[m0 + tt] * t.rows + r];
            const float4 c = u[tt];
            // (x.x + i x.y)(c.re + i c.im), x exact in FP32
            df_acc1(sr, lr, x.x, c.x, c.y);
            df_acc1(sr, lr, -x.y, c.z, c.w);
            df_acc1(si, li, x.x, c.z, c.w);
            df_acc1(si, li, x.y, c.x, c.y);
        }
        const float2 fr = df_fin(sr, lr), fi = df_fin(si, li);
        store_y(Y + t.yoff + jj * t.rows + r, fr.x, fr.y, fi.x, fi.y);
    }
}

// H_mu elements from double-float Y (the mixed builds): U_a^dagger Y and the
// projected exchange sum_g (v^1/2 P_i)_g conj(v^1/2 P_j)_g in double-float on
// the FP32 pipe; the diagonal term U_i^dagger diag(eps_c - eps_v) U_j on a
// shared orbit and W^div in FP64.  Pt: v^1/2-scaled projected exchange
// vectors in double-float (or null).
__global__ void project_left_df_kernel(DevBasis Bs, const TileTask* __restrict__ tiles, const float4* __restrict__ Y,
                                       const float4* __restrict__ Pt, int ng0, double xscale,
                                       const double* __restrict__ de, const double* __restrict__ w_div, double2* H,
                                       int64_t ld) {
    const TileTask t = tiles[blockIdx.z];
    const int64_t ii = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t nrow = t.ca1 - t.ca0, ncol = t.cb1 - t.cb0;
    if (ii >= nrow) return;
    const int64_t i = t.ca0 + ii;
    const int o = Bs.col_orbit[i];
    const int64_t m0 = Bs.orbit_off[o], n_o = Bs.orbit_off[o + 1] - m0;
    const float4* u = Bs.coef_df + Bs.col_off[i];
    for (int64_t jj = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; jj < ncol; jj += (int64_t)gridDim.y * blockDim.y) {
        const int64_t j = t.cb0 + jj;
        const float4* y = Y + t.yoff + jj * t.rows;
        // raw double-float sums, normalised once at the end
        float sr = 0.f, lr = 0.f, si = 0.f, li = 0.f;
#pragma unroll 4
        for (int64_t tt = 0; tt < n_o; ++tt) {
            const float4 a = u[tt], b = y[Bs.member_loc[m0 + tt]];   // conj(a) b
            df_acc(sr, lr, a.x, a.y, b.x, b.y);
            df_acc(sr, lr, a.z, a.w, b.z, b.w);
            df_acc(si, li, a.x, a.y, b.z, b.w);
            df_acc(si, li, -a.z, -a.w, b.x, b.y);
        }
        const float2 hr = df_fin(sr, lr), hi = df_fin(si, li);
        double2 h = make_double2((double)hr.x + (double)hr.y, (double)hi.x + (double)hi.y);
        if (de && Bs.col_orbit[j] == o) {
            const double2* ui = Bs.coef + Bs.col_off[i];
            const double2* uj = Bs.coef + Bs.col_off[j];
            double2 d = make_double2(0.0, 0.0);
            for (int64_t tt = 0; tt < n_o; ++tt) {
                double2 z = cmul(conjd(ui[tt]), uj[tt]);
                const double e = de[Bs.members[m0 + tt]];
                d.x = fma(e, z.x, d.x);
                d.y = fma(e, z.y, d.y);
            }
            h.x += d.x - (i == j ? *w_div : 0.0);
            h.y += d.y;
        }
        if (Pt) {
            const float4* pi = Pt + i * ng0;
            const float4* pj = Pt + j * ng0;
            float4 ex = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int g = 0; g < ng0; ++g) ex = cdf_dot_acc(ex, pj[g], pi[g]);   // P_i conj(P_j)
            const double2 e = cdf_to(ex);
            h.x = fma(xscale, e.x, h.x);
            h.y = fma(xscale, e.y, h.y);
        }
        H[j * ld + i] = h;
        if (t.star_a != t.star_b) H[i * ld + j] = conjd(h);
    }
}

__global__ void scale_to_df_kernel(const double2* __restrict__ P, const double* __restrict__ vbar, int64_t n, int ng0,
                                   float4* out) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n * ng0) return;
    const double s = sqrt(vbar[id % ng0]);
    const double2 p = P[id];
    out[id] = cdf_from(make_double2(s * p.x, s * p.y));
}

int launch_exchange_df(const double2* Pmu, const double* vbar, int64_t n, int ng0, float4* out, cudaStream_t st) {
    if (n == 0 || ng0 == 0) return BSE_OK;
    scale_to_df_kernel<<<(unsigned)ceil_div(n * ng0, 256), 256, 0, st>>>(Pmu, vbar, n, ng0, out);
    LAUNCH_CHECK();
    return BSE_OK;
}

__global__ void to_df_kernel(const double2* __restrict__ in, float4* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cdf_from(in[i]);
}

int launch_to_df(const double2* in, float4* out, int64_t n, cudaStream_t st) {
    if (n == 0) return BSE_OK;
    to_df_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(in, out, n);
    LAUNCH_CHECK();
    return BSE_OK;
}

__global__ void project_left_kernel(DevBasis Bs, const TileTask* __restrict__ tiles, const double2* __restrict__ Y,
                                    const double2* __restrict__ Pmu, const double* __restrict__ vbar, int ng0,
                                    double xscale, const double* __restrict__ de,
                                    const double* __restrict__ w_div, double2* H, int64_t ld) {
    const TileTask t = tiles[blockIdx.z];
    const int64_t ii = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t nrow = t.ca1 - t.ca0, ncol = t.cb1 - t.cb0;
    if (ii >= nrow) return;
    const int64_t i = t.ca0 + ii;
    const int o = Bs.col_orbit[i];
    const int64_t m0 = Bs.orbit_off[o], n_o = Bs.orbit_off[o + 1] - m0;
    const double2* u = Bs.coef + Bs.col_off[i];
    for (int64_t jj = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; jj < ncol; jj += (int64_t)gridDim.y * blockDim.y) {
        const int64_t j = t.cb0 + jj;
        const double2* y = Y + t.yoff + jj * t.rows;
        double2 acc = make_double2(0.0, 0.0);
        for (int64_t tt = 0; tt < n_o; ++tt) cfma_conj(acc, u[tt], y[Bs.member_loc[m0 + tt]]);
        if (de && Bs.col_orbit[j] == o) {
            // U_i^dagger diag(eps_c - eps_v) U_j on the shared orbit, minus W^div delta_ij (FP64)
            const double2* uj = Bs.coef + Bs.col_off[j];
            double2 d = make_double2(0.0, 0.0);
            for (int64_t tt = 0; tt < n_o; ++tt) {
                double2 z = cmul(conjd(u[tt]), uj[tt]);
                const double e = de[Bs.members[m0 + tt]];
                d.x = fma(e, z.x, d.x);
                d.y = fma(e, z.y, d.y);
            }
            acc.x += d.x - (i == j ? *w_div : 0.0);
            acc.y += d.y;
        }
        if (Pmu) {
            const double2* pi = Pmu + i * ng0;
            const double2* pj = Pmu + j * ng0;
            double2 ex = make_double2(0.0, 0.0);
            for (int g = 0; g < ng0; ++g) {
                double2 z = cmul(pi[g], conjd(pj[g]));
                ex.x = fma(vbar[g], z.x, ex.x);
                ex.y = fma(vbar[g], z.y, ex.y);
            }
            acc.x = fma(xscale, ex.x, acc.x);
            acc.y = fma(xscale, ex.y, acc.y);
        }
        H[j * ld + i] = acc;
        if (t.star_a != t.star_b) H[i * ld + j] = conjd(acc);
    }
}

int launch_project_right(const DevBasis& b, const TileTask* tiles, int ntiles, int x32, const void* X, double2* Y,
                         int64_t max_rows, int64_t max_cols, cudaStream_t st, int ydf) {
    if (ntiles == 0) return BSE_OK;
    dim3 blk(32, 8);
    int gy = ceil_div(max_cols, 8);
    if (gy > 64) gy = 64;
    if (gy < 1) gy = 1;
    for (int off = 0; off < ntiles; off += 65535) {
        int n = ntiles - off < 65535 ? ntiles - off : 65535;
        dim3 grd(ceil_div(max_rows, 32), gy, n);
        if (x32 && ydf)
            project_right_df_kernel<float4><<<grd, blk, 0, st>>>(b, tiles + off, (const float2*)X, (float4*)Y);
        else if (x32)
            project_right_df_kernel<double2><<<grd, blk, 0, st>>>(b, tiles + off, (const float2*)X, Y);
        else
            project_right_kernel<double2><<<grd, blk, 0, st>>>(b, tiles + off, (const double2*)X, Y);
        LAUNCH_CHECK();
    }
    return BSE_OK;
}

int launch_project_left(const DevBasis& b, const TileTask* tiles, int ntiles, const double2* Y, const double2* Pmu,
                        const double* vbar, int ng0, double xscale, const double* de, const double* w_div, double2* H,
                        int64_t ld, int64_t max_ca, int64_t max_cb, cudaStream_t st, int ydf, const float4* Pt) {
    if (ntiles == 0) return BSE_OK;
    dim3 blk(32, 8);
    int gy = ceil_div(max_cb, 8);
    if (gy > 64) gy = 64;
    if (gy < 1) gy = 1;
    for (int off = 0; off < ntiles; off += 65535) {
        int n = ntiles - off < 65535 ? ntiles - off : 65535;
        dim3 grd(ceil_div(max_ca, 32) > 0 ? ceil_div(max_ca, 32) : 1, gy, n);
        if (ydf)
            project_left_df_kernel<<<grd, blk, 0, st>>>(b, tiles + off, (const float4*)Y, Pmu ? Pt : nullptr, ng0,
                                                        xscale, de, w_div, H, ld);
        else
            project_left_kernel<<<grd, blk, 0, st>>>(b, tiles + off, Y, Pmu, vbar, ng0, xscale, de, w_div, H, ld);
        LAUNCH_CHECK();
    }
    return BSE_OK;
}

// Pmu[i][g] = sum_t conj(U_i[t]) P[member_t][g]
__global__ void exchange_project_kernel(DevBasis Bs, const double2* __restrict__ P, int ng0, double2* Pmu) {
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= Bs.dim * ng0) return;
    int64_t i = id / ng0;
    int g = (int)(id % ng0);
    const int o = Bs.col_orbit[i];
    const int64_t m0 = Bs.orbit_off[o], n_o = Bs.orbit_off[o + 1] - m0;
    const double2* u = Bs.coef + Bs.col_off[i];
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t tt = 0; tt < n_o; ++tt) cfma_conj(acc, u[tt], P[Bs.members[m0 + tt] * ng0 + g]);
    Pmu[id] = acc;
}

int launch_exchange_project(const DevBasis& b, const double2* P, int ng0, double2* Pmu, cudaStream_t st) {
    int64_t n = b.dim * ng0;
    if (n == 0) return BSE_OK;
    exchange_project_kernel<<<ceil_div(n, 256), 256, 0, st>>>(b, P, ng0, Pmu);
    LAUNCH_CHECK();
    return BSE_OK;
}

// H[I, J] += xscale sum_g vbar_g P[I][g] conj(P[J][g])  (column-major H)
__global__ void exchange_full_kernel(const double2* __restrict__ P, const double* __restrict__ vbar, int ng0,
                                     int64_t N, double xscale, double2* H, int64_t ld) {
    int64_t I = (int64_t)blockIdx.x * 32 + threadIdx.x;
    int64_t J = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (I >= N || J >= N) return;
    double2 ex = make_double2(0.0, 0.0);
    for (int g = 0; g < ng0; ++g) {
        double2 z = cmul(P[I * ng0 + g], conjd(P[J * ng0 + g]));
        ex.x = fma(vbar[g], z.x, ex.x);
        ex.y = fma(vbar[g], z.y, ex.y);
    }
    double2 h = H[J * ld + I];
    h.x = fma(xscale, ex.x, h.x);
    h.y = fma(xscale, ex.y, h.y);
    H[J * ld + I] = h;
}

int launch_exchange_full(const double2* P, const double* vbar, int ng0, int64_t N, double xscale, double2* H,
                         int64_t ld, cudaStream_t st) {
    dim3 blk(32, 8), grd(ceil_div(N, 32), ceil_div(N, 8));
    exchange_full_kernel<<<grd, blk, 0, st>>>(P, vbar, ng0, N, xscale, H, ld);
    LAUNCH_CHECK();
    return BSE_OK;
}

// H[I, I] += eps_c - eps_v - W^div (column-major H)
__global__ void diag_full_kernel(const double* __restrict__ de, int64_t N, const double* __restrict__ w_div, double2* H,
                                 int64_t ld) {
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I < N) H[I * ld + I].x += de[I] - *w_div;
}

int launch_diag_full(const double* de, int64_t N, const double* w_div, double2* H, int64_t ld, cudaStream_t st) {
    diag_full_kernel<<<ceil_div(N, 256), 256, 0, st>>>(de, N, w_div, H, ld);
    LAUNCH_CHECK();
    return BSE_OK;
}

__global__ void basis_dense_kernel(DevBasis Bs, double2* U, int64_t ld) {
    int64_t j = blockIdx.x;
    if (j >= Bs.dim) return;
    const int o = Bs.col_orbit[j];
    const int64_t m0 = Bs.orbit_off[o], n_o = Bs.orbit_off[o + 1] - m0;
    for (int64_t tt = threadIdx.x; tt < n_o; tt += blockDim.x) U[j * ld + Bs.members[m0 + tt]] = Bs.coef[Bs.col_off[j] + tt];
}

int launch_basis_dense(const DevBasis& b, double2* U, int64_t ld, cudaStream_t st) {
    if (b.dim == 0) return BSE_OK;
    basis_dense_kernel<<<(unsigned)b.dim, 64, 0, st>>>(b, U, ld);
    LAUNCH_CHECK();
    return BSE_OK;
}

// ---------------------------------------------------------------------------
// spectrum (Eqs. oscillator, oscillatorA, reducible_polar)
// ---------------------------------------------------------------------------
__global__ void dipoles_kernel(DevSys S, double2* Bout) {
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int nv = S.nv, nc = S.nc;
    if (id >= (int64_t)S.nk * nv * nc) return;
    int k = (int)(id / (nv * nc)), v = (int)((id / nc) % nv), c = (int)(id % nc);
    const double2* cv = S.coef + ((int64_t)k * S.nb + v) * S.npw_max;
    const double2* cc = S.coef + ((int64_t)k * S.nb + nv + c) * S.npw_max;
    const double f[3] = {S.kidx[3 * k] / (double)S.n1, S.kidx[3 * k + 1] / (double)S.n2,
                         S.kidx[3 * k + 2] / (double)S.n3};
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < S.npw[k]; ++i) {
        const int* m = S.gk + ((int64_t)k * S.npw_max + i) * 3;
        double qp = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double pa = 0.0;
#pragma unroll
            for (int b = 0; b < 3; ++b) pa += S.recip[3 * a + b] * (f[b] + m[b]);
            qp += S.qhat[a] * pa;
        }
        double2 z = cc[i];
        z.x *= qp;
        z.y *= qp;
        cfma_conj(acc, cv[i], z);
    }
    double de = S.eps[k * S.nb + nv + c] - S.scissor - S.eps[k * S.nb + v];
    double sc = 1.0 / (sqrt(S.v_uc) * de);
    Bout[id] = make_double2(acc.x * sc, acc.y * sc);
}

int launch_dipoles(const DevSys& s, double2* B, cudaStream_t st) {
    int64_t n = (int64_t)s.nk * s.nv * s.nc;
    dipoles_kernel<<<ceil_div(n, 128), 128, 0, st>>>(s, B);
    LAUNCH_CHECK();
    return BSE_OK;
}

__global__ void bmu_kernel(DevBasis Bs, const double2* __restrict__ B, double2* Bmu) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Bs.dim) return;
    const int o = Bs.col_orbit[j];
    const int64_t m0 = Bs.orbit_off[o], n_o = Bs.orbit_off[o + 1] - m0;
    const double2* u = Bs.coef + Bs.col_off[j];
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t tt = 0; tt < n_o; ++tt) cfma(acc, u[tt], B[Bs.members[m0 + tt]]);
    Bmu[j] = acc;
}

int launch_bmu(const DevBasis& b, const double2* B, double2* Bmu, cudaStream_t st) {
    if (b.dim == 0) return BSE_OK;
    bmu_kernel<<<ceil_div(b.dim, 128), 128, 0, st>>>(b, B, Bmu);
    LAUNCH_CHECK();
    return BSE_OK;
}

// osc[l] = sum_p |sum_i a[i, l] Bmu[p][i]|^2, one warp per eigenvector
__global__ void oscillator_kernel(const double2* __restrict__ a, int64_t lda, int64_t dim,
                                  const double2* __restrict__ Bmu, int nparts, double* osc) {
    int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (l >= dim) return;
    double tot = 0.0;
    for (int p = 0; p < nparts; ++p) {
        double2 acc = make_double2(0.0, 0.0);
        for (int64_t i = lane; i < dim; i += 32) cfma(acc, a[l * lda + i], Bmu[(int64_t)p * dim + i]);
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        tot += acc.x * acc.x + acc.y * acc.y;
    }
    if (lane == 0) osc[l] = tot;
}

int launch_oscillators(const double2* a, int64_t lda, int64_t dim, const double2* Bmu, int nparts, double* osc,
                       cudaStream_t st) {
    if (dim == 0) return BSE_OK;
    oscillator_kernel<<<ceil_div(dim * 32, 256), 256, 0, st>>>(a, lda, dim, Bmu, nparts, osc);
    LAUNCH_CHECK();
    return BSE_OK;
}

// Im eps_M on the frequency grid: 8 lanes per frequency share the sum over
// the levels (one warp per frequency would leave the FP64 pipes of most SM
// sub-partitions idle at a few thousand frequencies); Newton reciprocals.
constexpr int kSpecLanes = 8;
__global__ void spectrum_kernel(const double* __restrict__ Om, const double* __restrict__ osc, int64_t dim,
                                const double* __restrict__ omega, int64_t n_omega, double eta, double pref,
                                double* im) {
    // the Lorentzian terms in double-float on the FP32 pipe (GB300's FP64
    // pipe is 64 times narrower); the levels and weights are read in FP64
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t w = g / kSpecLanes;
    const int part = (int)(g % kSpecLanes);
    const float2 x = df_from(w < n_omega ? omega[w] : 0.0);
    const float2 e2 = df_from(eta * eta);
    float sh = 0.f, sl = 0.f;
    if (w < n_omega)
        for (int64_t l = part; l < dim; l += kSpecLanes) {
            const float2 om = df_from(__ldg(Om + l)), ow = df_from(__ldg(osc + l));
            const float2 d1 = df_add(x, df_neg(om)), d2 = df_add(x, om);
            float a = e2.x, al = e2.y, b = e2.x, bl = e2.y;
            df_acc(a, al, d1.x, d1.y, d1.x, d1.y);
            df_acc(b, bl, d2.x, d2.y, d2.x, d2.y);
            const float2 r = df_add(df_rcp(df_fin(a, al)), df_neg(df_rcp(df_fin(b, bl))));
            df_acc(sh, sl, ow.x, ow.y, r.x, r.y);
            const float2 f = df_fin(sh, sl);
            sh = f.x;
            sl = f.y;
        }
    double acc = (double)sh + (double)sl;
#pragma unroll
    for (int o = kSpecLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (part == 0 && w < n_omega) im[w] = pref * eta * acc;
}

int launch_spectrum(const double* Om, const double* osc, int64_t dim, const double* omega, int64_t n_omega, double eta,
                    double pref, double* im, cudaStream_t st) {
    if (n_omega == 0) return BSE_OK;
    spectrum_kernel<<<ceil_div(n_omega * kSpecLanes, 256), 256, 0, st>>>(Om, osc, dim, omega, n_omega, eta, pref, im);
    LAUNCH_CHECK();
    return BSE_OK;
}

// ---------------------------------------------------------------------------
// head correction: smoothed double-counting sum of Eq. divergence_sum over
// Q = sum_j X_j b_j / n_j (X integer, Q != 0), one thread per (X1, X2) column
// ---------------------------------------------------------------------------
constexpr int kWdivMaxOps = 48;
struct WdivSym {
    int nops;
    int M[kWdivMaxOps][9];      // action on the integer coordinates X, row-major
    float u[kWdivMaxOps][3];    // p - M_g^T p (the identity's row is zero)
    float inv3[kWdivMaxOps];    // 1 / u[g][2], or 0 when |u[g][2]| is negligible
    double p[3];                // generic projection vector
};

struct WdivGeom {
    double s[9];      // columns: b_j / n_j (row-major 3x3)
    double L[9];
    double b, qmax, delta, lim;
    int e1, e2;
};

__global__ void wdiv_kernel(WdivGeom g, double* partial) {
    __shared__ double red[256];
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t ncol = (int64_t)(2 * g.e1 + 1) * (2 * g.e2 + 1);
    double acc = 0.0;
    if (id < ncol) {
        int x1 = (int)(id / (2 * g.e2 + 1)) - g.e1;
        int x2 = (int)(id % (2 * g.e2 + 1)) - g.e2;
        double p[3], s3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            p[a] = g.s[3 * a] * x1 + g.s[3 * a + 1] * x2;
            s3[a] = g.s[3 * a + 2];
        }
        // |p + x3 s3|^2 <= lim^2: quadratic in x3
        double A = s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2];
        double Bq = 2.0 * (p[0] * s3[0] + p[1] * s3[1] + p[2] * s3[2]);
        double C = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] - g.lim * g.lim;
        double disc = Bq * Bq - 4.0 * A * C;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            int lo = (int)floor((-Bq - sq) / (2.0 * A)) - 1;
            int hi = (int)ceil((-Bq + sq) / (2.0 * A)) + 1;
            // Along the line x3 the quadratics q^2 = |p + x3 s3|^2 and Q^T L Q advance
            // by forward differences and exp(-b q^2) by the exact recurrence
            //   E(x3 + 1) = E(x3) R(x3),  R(x3 + 1) = R(x3) C,  C = exp(-2 b |s3|^2),
            // all restarted from their definitions every 64 points to bound the
            // rounding growth; 1/(Q^T L Q) by a Newton reciprocal (no FP64 divide).
            const double C2 = exp(-2.0 * g.b * A);
            const double lim2 = g.lim * g.lim, in2 = (g.qmax - g.delta) * (g.qmax - g.delta);
            double Ls[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) Ls[a] = g.L[3 * a] * s3[0] + g.L[3 * a + 1] * s3[1] + g.L[3 * a + 2] * s3[2];
            const double sLs = s3[0] * Ls[0] + s3[1] * Ls[1] + s3[2] * Ls[2];
            double E = 0.0, Rr = 0.0, q2 = 0.0, dq2 = 0.0, ql = 0.0, dql = 0.0;
            for (int x3 = lo; x3 <= hi; ++x3) {
                if (((x3 - lo) & 63) == 0) {
                    const double Q[3] = {p[0] + x3 * s3[0], p[1] + x3 * s3[1], p[2] + x3 * s3[2]};
                    q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
                    dq2 = 2.0 * (Q[0] * s3[0] + Q[1] * s3[1] + Q[2] * s3[2]) + A;
                    ql = 0.0;
                    double QLs = 0.0, sLQ = 0.0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            ql += Q[a] * g.L[3 * a + c] * Q[c];
                            sLQ += s3[a] * g.L[3 * a + c] * Q[c];
                        }
                        QLs += Q[a] * Ls[a];
                    }
                    dql = QLs + sLQ + sLs;
                    E = exp(-g.b * q2);
                    Rr = exp(-g.b * dq2);
                } else {
                    q2 += dq2;
                    dq2 += 2.0 * A;
                    ql += dql;
                    dql += 2.0 * sLs;
                    E *= Rr;
                    Rr *= C2;
                }
                if ((x1 == 0 && x2 == 0 && x3 == 0) || q2 > lim2) continue;
                double w = 1.0;
                if (q2 >= in2) {
                    double x = (sqrt(q2) - g.qmax) / g.delta;
                    if (x > 1.0) continue;
                    w = (x * x * x - 3.0 * x + 2.0) * 0.25;
                }
                acc = fma(E * w, rcp_nr(ql), acc);
            }
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// The same sum over one representative per orbit of the point group: the
// summand depends on Q only through |Q| and Q^T L Q, both invariant when L
// is, so sum_Q f(Q) = sum_{representatives} |orbit| f(Q).  Q = sum_j X_j b_j /
// n_j with X integer; the group acts on X by integer matrices M_g.  X is the
// representative of its orbit when its projection X.p on a generic vector p
// is the largest over the orbit (ties, possible only for distinct points with
// equal projections, by the lexicographic order of the integer vectors); its
// orbit has |G| / |stab(X)| points.  The necessary conditions (p - M_g^T p).X
// >= 0 are linear in X_3, so each column (X_1, X_2) is clipped to the
// interval of its cone (wdiv_clip_kernel); after a scan of the counts every
// column knows the index of its first candidate (wdiv_offsets_kernel), and
// the candidates are evaluated one per thread (wdiv_point_kernel, which finds
// a candidate's column by binary search over those offsets).  That keeps the
// FP64 work of the ~1/|G| remaining points free of the columns' very uneven
// lengths, and the whole sum runs without a host round trip.
struct WdivCols {
    int* lo;            // [ncol] first X_3 of the column's interval
    int* cnt;           // [ncol] candidates of the column
    int64_t* blocksum;  // [nblk] candidates per block of 256 columns, then their exclusive scan
    int64_t* total;     // [1]
    int64_t* off;       // [ncol] index of the column's first candidate (nondecreasing)
};

__device__ __forceinline__ void wdiv_column(const WdivGeom& g, const WdivSym& sy, int64_t id, int& lo, int& hi) {
    const int x1 = (int)(id / (2 * g.e2 + 1)) - g.e1;
    const int x2 = (int)(id % (2 * g.e2 + 1)) - g.e2;
    double p[3], s3[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p[a] = g.s[3 * a] * x1 + g.s[3 * a + 1] * x2;
        s3[a] = g.s[3 * a + 2];
    }
    const double A = s3[0] * s3[0] + s3[1] * s3[1] + s3[2] * s3[2];
    const double Bq = 2.0 * (p[0] * s3[0] + p[1] * s3[1] + p[2] * s3[2]);
    const double C = p[0] * p[0] + p[1] * p[1] + p[2] * p[2] - g.lim * g.lim;
    const double disc = Bq * Bq - 4.0 * A * C;
    lo = 0;
    hi = -1;
    if (disc < 0.0) return;
    const double sq = sqrt(disc);
    lo = (int)floor((-Bq - sq) / (2.0 * A)) - 1;
    hi = (int)ceil((-Bq + sq) / (2.0 * A)) + 1;
    // clip to the cone u_g . X >= 0 (FP32 with two points of slack; exact checks follow)
    for (int o = 0; o < sy.nops && lo <= hi; ++o) {
        const float b0 = sy.u[o][0] * (float)x1 + sy.u[o][1] * (float)x2;
        const float ia = sy.inv3[o];
        if (ia == 0.0f) {
            if (b0 < -1e-2f) hi = lo - 1;
        } else {
            const float t = -b0 * ia;
            if (sy.u[o][2] > 0.0f) lo = max(lo, (int)floorf(t) - 2);
            else hi = min(hi, (int)ceilf(t) + 2);
        }
    }
}

__global__ void wdiv_clip_kernel(WdivGeom g, const __grid_constant__ WdivSym sy, WdivCols c) {
    __shared__ int64_t red[256];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ncol = (int64_t)(2 * g.e1 + 1) * (2 * g.e2 + 1);
    int n = 0;
    if (id < ncol) {
        int lo, hi;
        wdiv_column(g, sy, id, lo, hi);
        n = hi >= lo ? hi - lo + 1 : 0;
        c.lo[id] = lo;
        c.cnt[id] = n;
    }
    red[threadIdx.x] = n;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) c.blocksum[blockIdx.x] = red[0];
}

// exclusive scan of the block sums (one block)
__global__ void wdiv_scan_kernel(WdivCols c, int64_t nblk) {
    __shared__ int64_t s[1024];
    const int t = threadIdx.x;
    const int64_t per = (nblk + 1023) / 1024;
    const int64_t i0 = t * per, i1 = min(nblk, i0 + per);
    int64_t loc = 0;
    for (int64_t i = i0; i < i1; ++i) loc += c.blocksum[i];
    s[t] = loc;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = t >= off ? s[t - off] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    int64_t run = s[t] - loc;
    for (int64_t i = i0; i < i1; ++i) {
        const int64_t x = c.blocksum[i];
        c.blocksum[i] = run;
        run += x;
    }
    if (t == 1023) *c.total = s[1023];
}

__global__ void wdiv_offsets_kernel(WdivGeom g, WdivCols c) {
    __shared__ int s[256];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ncol = (int64_t)(2 * g.e1 + 1) * (2 * g.e2 + 1);
    const int n = id < ncol ? c.cnt[id] : 0;
    s[threadIdx.x] = n;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const int v = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    if (id < ncol) c.off[id] = c.blocksum[blockIdx.x] + s[threadIdx.x] - n;
}

// one candidate per thread, grid-stride over the total; partial sums per block
__global__ void wdiv_point_kernel(WdivGeom g, const __grid_constant__ WdivSym sy, WdivCols c, double* partial) {
    __shared__ double red[256];
    const int64_t total = *c.total;
    const int64_t ncol = (int64_t)(2 * g.e1 + 1) * (2 * g.e2 + 1);
    const double lim2 = g.lim * g.lim, in2 = (g.qmax - g.delta) * (g.qmax - g.delta);
    double acc = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        // the column holding candidate q: the last one whose first candidate is <= q
        // (an empty column shares its offset with the next column, so it is never last)
        int64_t lo = 0, hi = ncol - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(c.off + mid) <= q) lo = mid;
            else hi = mid - 1;
        }
        const int64_t id = lo;
        const int x1 = (int)(id / (2 * g.e2 + 1)) - g.e1;
        const int x2 = (int)(id % (2 * g.e2 + 1)) - g.e2;
        const int x3 = __ldg(c.lo + id) + (int)(q - __ldg(c.off + id));
        if (x1 == 0 && x2 == 0 && x3 == 0) continue;
        double Q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) Q[a] = g.s[3 * a] * x1 + g.s[3 * a + 1] * x2 + g.s[3 * a + 2] * x3;
        const double q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
        if (q2 > lim2) continue;
        // cone values in FP32: all clearly positive means an interior point, whose
        // stabiliser is trivial (orbit of |G| points); any clearly negative one rejects
        float vmin = 1e30f;
        for (int o = 0; o < sy.nops; ++o) {
            if (sy.u[o][0] == 0.0f && sy.u[o][1] == 0.0f && sy.u[o][2] == 0.0f) continue;   // the identity
            vmin = fminf(vmin, sy.u[o][0] * (float)x1 + sy.u[o][1] * (float)x2 + sy.u[o][2] * (float)x3);
        }
        if (vmin < -1e-2f) continue;
        int mult = sy.nops;
        if (vmin <= 1e-2f) {   // near a face: exact test on the integer coordinates
            const double pX = sy.p[0] * x1 + sy.p[1] * x2 + sy.p[2] * x3;
            int stab = 0;
            bool rep = true;
            for (int o = 0; o < sy.nops; ++o) {
                const int* M = sy.M[o];
                const int y0 = M[0] * x1 + M[1] * x2 + M[2] * x3;
                const int y1 = M[3] * x1 + M[4] * x2 + M[5] * x3;
                const int y2 = M[6] * x1 + M[7] * x2 + M[8] * x3;
                if (y0 == x1 && y1 == x2 && y2 == x3) {
                    ++stab;
                    continue;
                }
                const double pY = sy.p[0] * y0 + sy.p[1] * y1 + sy.p[2] * y2;
                if (pY > pX || (pY == pX && (y0 > x1 || (y0 == x1 && (y1 > x2 || (y1 == x2 && y2 > x3)))))) {
                    rep = false;
                    break;
                }
            }
            if (!rep) continue;
            mult = sy.nops / stab;
        }
        double w = (double)mult;
        if (q2 >= in2) {
            const double x = (sqrt(q2) - g.qmax) / g.delta;
            if (x > 1.0) continue;
            w *= (x * x * x - 3.0 * x + 2.0) * 0.25;
        }
        double ql = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) ql += Q[a] * g.L[3 * a + cc] * Q[cc];
        acc = fma(exp(-g.b * q2) * w, rcp_nr(ql), acc);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// fixed-order reduction of the block partials (deterministic)
__global__ void reduce_kernel(const double* __restrict__ partial, int64_t n, double* out) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void wdiv_finalize_kernel(const double* __restrict__ sum, double a, double b, double* w) {
    *w = a - b * *sum;
}

int launch_wdiv_finalize(const double* sum, double a, double b, double* w, cudaStream_t st) {
    wdiv_finalize_kernel<<<1, 1, 0, st>>>(sum, a, b, w);
    LAUNCH_CHECK();
    return BSE_OK;
}

// extent of the integer coordinates X_j of the points Q = sum_j X_j b_j / n_j
// with |Q| <= lim (clamped far above any mesh that is accepted, so that the
// conversion cannot overflow)
static void wdiv_extent(const double* lattice, const int* n, double lim, int e[3]) {
    for (int j = 0; j < 3; ++j) {
        double len = sqrt(lattice[j] * lattice[j] + lattice[3 + j] * lattice[3 + j] + lattice[6 + j] * lattice[6 + j]);
        const double x = ceil((double)n[j] * lim * len / (2.0 * M_PI)) + 1.0;
        e[j] = x < (double)(1 << 28) ? (int)x : (1 << 28);
    }
}

int64_t wdiv_column_length(const double* lattice, const int* n, double qmax, double delta) {
    int e[3];
    wdiv_extent(lattice, n, qmax + delta, e);
    return 2 * (int64_t)e[2] + 1;
}

size_t wdiv_sym_bytes(const double* lattice, const int* n, double qmax, double delta) {
    int e[3];
    wdiv_extent(lattice, n, qmax + delta, e);
    const int64_t ncol = (int64_t)(2 * e[0] + 1) * (2 * e[1] + 1);
    const int64_t nblk = (ncol + 255) / 256;
    return sizeof(int) * 2 * (size_t)ncol + 16 + sizeof(int64_t) * (size_t)(nblk + 1 + ncol);
}

int64_t wdiv_partials(const double* lattice, const int* n, double qmax, double delta) {
    int e[3];
    wdiv_extent(lattice, n, qmax + delta, e);
    int64_t ncol = (int64_t)(2 * e[0] + 1) * (2 * e[1] + 1);
    return (ncol + 255) / 256;
}

int launch_wdiv(const double* recip_and_lattice, const int* n, const double* L, double b, double qmax, double delta,
                double* partial, int64_t npartial_max, double* out, cudaStream_t st, int nops, const int* Mx,
                WdivScratch* sym_scratch) {
    // recip_and_lattice: 18 doubles, reciprocal basis then lattice (row-major)
    WdivGeom g;
    const double* recip = recip_and_lattice;
    const double* lattice = recip_and_lattice + 9;
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 3; ++j) g.s[3 * a + j] = recip[3 * a + j] / n[j];
    for (int i = 0; i < 9; ++i) g.L[i] = L[i];
    g.b = b;
    g.qmax = qmax;
    g.delta = delta;
    g.lim = qmax + delta;
    int e[3];
    wdiv_extent(lattice, n, g.lim, e);
    g.e1 = e[0];
    g.e2 = e[1];
    int64_t ncol = (int64_t)(2 * e[0] + 1) * (2 * e[1] + 1);
    int64_t nblk = (ncol + 255) / 256;
    if (nblk > npartial_max) return fail(BSE_EINVAL, "head-correction scratch too small (%lld > %lld)",
                                         (long long)nblk, (long long)npartial_max);
    if (nops > 0 && nops <= kWdivMaxOps && Mx && sym_scratch) {
        WdivSym sy;
        sy.nops = nops;
        // a generic direction (no small-integer relation among the components)
        sy.p[0] = 1.0;
        sy.p[1] = 0.7548776662466927;   // plastic-number ratios
        sy.p[2] = 0.5698402909980532;
        for (int o = 0; o < nops; ++o) {
            for (int i = 0; i < 9; ++i) sy.M[o][i] = Mx[9 * o + i];
            for (int j = 0; j < 3; ++j) {
                double mtp = 0.0;   // (M^T p)_j
                for (int i = 0; i < 3; ++i) mtp += Mx[9 * o + 3 * i + j] * sy.p[i];
                const double u = sy.p[j] - mtp;
                sy.u[o][j] = std::fabs(u) < 1e-12 ? 0.0f : (float)u;
            }
            sy.inv3[o] = std::fabs(sy.u[o][2]) < 1e-6f ? 0.0f : 1.0f / sy.u[o][2];
        }
        WdivCols c;
        char* ptr = (char*)sym_scratch->base;
        c.lo = (int*)ptr;
        c.cnt = c.lo + ncol;
        c.blocksum = (int64_t*)(((uintptr_t)(c.cnt + ncol) + 15) & ~(uintptr_t)15);
        c.total = c.blocksum + nblk;
        c.off = c.total + 1;
        wdiv_clip_kernel<<<(unsigned)nblk, 256, 0, st>>>(g, sy, c);
        LAUNCH_CHECK();
        wdiv_scan_kernel<<<1, 1024, 0, st>>>(c, nblk);
        LAUNCH_CHECK();
        wdiv_offsets_kernel<<<(unsigned)nblk, 256, 0, st>>>(g, c);
        LAUNCH_CHECK();
        const int64_t pb = std::min<int64_t>(nblk, 152 * 8);
        wdiv_point_kernel<<<(unsigned)pb, 256, 0, st>>>(g, sy, c, partial);
        LAUNCH_CHECK();
        reduce_kernel<<<1, 1024, 0, st>>>(partial, pb, out);
        LAUNCH_CHECK();
        return BSE_OK;
    } else {
        wdiv_kernel<<<(unsigned)nblk, 256, 0, st>>>(g, partial);
    }
    LAUNCH_CHECK();
    reduce_kernel<<<1, 1024, 0, st>>>(partial, nblk, out);
    LAUNCH_CHECK();
    return BSE_OK;
}

// ---------------------------------------------------------------------------
// algorithmic work: n_ovl(k,k') = #{(p', Q): p' in S_k', Q in S_q, p' + Q in S_k}
// ---------------------------------------------------------------------------
__global__ void count_overlap_kernel(DevSys S, const PairTask* __restrict__ tasks, unsigned long long* out) {
    __shared__ unsigned long long red[256];
    const PairTask t = tasks[blockIdx.x];
    int fold[3];
    const int q = mesh_minus(S, t.k, t.kp, fold);
    const int ng = S.ng[q], npkp = S.npw[t.kp];
    const int* gq = S.gq + (int64_t)q * S.ng_max * 3;
    const int* gk = S.gk + (int64_t)t.kp * S.npw_max * 3;
    unsigned long long c = 0;
    for (int e = threadIdx.x; e < ng * npkp; e += blockDim.x) {
        int g = e / npkp, j = e % npkp;
        c += sphere_index(S, t.k, gk[3 * j] + gq[3 * g] + fold[0], gk[3 * j + 1] + gq[3 * g + 1] + fold[1],
                          gk[3 * j + 2] + gq[3 * g + 2] + fold[2]) >= 0;
    }
    red[threadIdx.x] = c;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

int launch_count_overlap(const DevSys& s, const PairTask* tasks, int64_t ntasks, unsigned long long* out,
                         cudaStream_t st) {
    for (int64_t off = 0; off < ntasks; off += 1 << 30) {
        int64_t n = ntasks - off < (1 << 30) ? ntasks - off : (1 << 30);
        count_overlap_kernel<<<(unsigned)n, 256, 0, st>>>(s, tasks + off, out);
        LAUNCH_CHECK();
    }
    return BSE_OK;
}

}  // namespace bse
