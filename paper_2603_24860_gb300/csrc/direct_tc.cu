// Direct term with the dense contractions on the 5th-generation tensor
// cores (tcgen05), in split precision: every operand x is stored as
// hi = e(x), lo = e(x - hi) in a 16-bit type e (bf16 or fp16), and a product
// A B is formed as A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in
// TMEM.  bf16 keeps FP32's exponent range with 2 x 8 significant bits; fp16
// keeps 2 x 11 bits but overflows above 65504 and loses bits below 2^-14, so
// every operand is scaled by a power of two that brings its largest element
// to [2^13, 2^14): W(q) per q, the pair densities per k pair, T per CTA.  The
// scales are exact and are divided out in the epilogue; both types use them.
//
//   rho_nn'(k,k';Q) = sum_{p'} conj(c_kn(p' + Q)) c_k'n'(p')   (CUDA cores, FP32; Eq. w_interaction)
//   T = W(q) conj(rho_vv')         MMA1, all pairs of a group share W(q)
//   K^d = 1/V rho_cc'^T T          MMA2, one pair at a time           (Eq. BSE-eigval)
//
// One CTA per group of up to 4 k pairs with the same q = k - k' (fewer when
// the operands of larger spheres fill shared memory or TMEM).  Complex
// products use real operands:
//   MMA1  T_r = Wr rho_r + Wi rho_i,  T_i = Wi rho_r + Wr (-rho_i)   (M = 128 rows Q, K = NGp)
//   MMA2  A2 = [[rho_r, -rho_i], [rho_i, rho_r]] (rows: Re K | Im K), B2 = [T_r | T_i]  (K = 2 NGp)
// so NG <= 128.  W(q) (Wr and Wi, hi and lo) is prepared once per q in the
// core-matrix layout and brought in by one bulk copy (from L2 as a rule) into
// the shared memory the pair densities were staged in; A2 and the epilogue
// staging reuse it after MMA1.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "grid_sync.h"
#include "internal.h"
#include "tc_ptx.h"

namespace bse {

using tc::core_off;

constexpr int kMaxG = 4;                            // pairs per group at most
constexpr int kSlots = 4;                           // band pairs per lane in the pair densities (nc^2 + nv^2 <= 128)
constexpr int kTmemCols = 256;                      // T_r, T_i and K^d of every pair: 3 nr kg columns
constexpr size_t kSmemBudget = 227 * 1024 - 2048;   // dynamic shared memory per CTA
constexpr size_t kSmemFloor = 82 * 1024;            // at most two CTAs (2 x 256 TMEM columns) per SM

struct TcPlan {
    size_t a, b, rc, st_coef, st_cnt, st_list, st_rho, total;   // a: W / A2 / epilogue and, before them, the staging
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 1023) & ~(size_t)1023; }
__host__ __device__ inline size_t zmax(size_t a, size_t b) { return a > b ? a : b; }
// rows of B1 and B2 per k pair: the nv^2 valence pairs padded to a multiple of 16 (N of MMA2)
__host__ __device__ inline int tc_rows(int nv) { return (nv * nv + 15) / 16 * 16; }

// ngp: NG padded to a multiple of 16 (K of MMA1); kg: pairs per group
__host__ __device__ inline TcPlan tc_plan(int kg, int ngp, int nb, int nv, int nc, int npw_max, int ng_max) {
    TcPlan p;
    const int nr = tc_rows(nv);
    const size_t a1 = (size_t)4 * 128 * ngp * 2;              // Wr hi, Wr lo, Wi hi, Wi lo: 128 x ngp each
    const size_t a2 = (size_t)2 * 128 * (2 * ngp) * 2;        // A2 hi, lo: 128 x 2 ngp each
    const size_t epi = (size_t)kg * nr * 128 * sizeof(float);
    p.st_coef = a16((size_t)npw_max * nb * sizeof(float2));
    p.st_cnt = a16((size_t)ng_max * sizeof(int));
    p.st_list = a16((size_t)ng_max * npw_max * sizeof(int));
    p.st_rho = a16((size_t)ng_max * (nc * nc + nv * nv) * sizeof(float2));
    const size_t staging = 2 * p.st_coef + p.st_cnt + p.st_list + p.st_rho;
    p.a = a16(zmax(zmax(zmax(a1, a2), epi), staging));
    const size_t b1 = (size_t)6 * kg * nr * ngp * 2;         // rho_r, rho_i, -rho_i (hi, lo): (nr kg) x ngp each
    const size_t b2 = (size_t)2 * kg * nr * (2 * ngp) * 2;   // [T_r | T_i] hi, lo: (nr kg) x 2 ngp each
    p.b = a16(zmax(b1, b2));
    p.rc = a16((size_t)kg * nc * nc * ngp * sizeof(float2));
    p.total = p.a + p.b + p.rc + 1024 + 64;
    return p;
}

// the 16-bit operand types: conversions and the instruction descriptor's type flag
template <typename E>
struct Elem;
template <>
struct Elem<__nv_bfloat16> {
    static constexpr int kBf16 = 1;
    static __device__ __forceinline__ __nv_bfloat16 from(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <>
struct Elem<__half> {
    static constexpr int kBf16 = 0;
    static __device__ __forceinline__ __half from(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float to(__half x) { return __half2float(x); }
};

template <typename E>
__device__ __forceinline__ void split16(float x, E& hi, E& lo) {
    hi = Elem<E>::from(x);
    lo = Elem<E>::from(x - Elem<E>::to(hi));
}

// exponent e with max_abs * 2^e in [2^13, 2^14) (0 for an all-zero operand), clamped to keep 2^e a normal float
__device__ __forceinline__ int scale_exp(float max_abs) {
    if (!(max_abs > 0.f)) return 0;
    int e = 13 - ilogbf(max_abs);
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// 2^e for |e| <= 126, built from the exponent field (exact)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// block-wide maximum of a non-negative float (bit patterns of non-negative floats order like integers)
__device__ __forceinline__ float block_max(float m, unsigned* s_slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(s_slot, __float_as_uint(m));
    __syncthreads();
    return __uint_as_float(*s_slot);
}

__device__ __forceinline__ void cmacc32(float2& acc, float2 a, float2 b) {   // acc += conj(a) * b
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

// Persistent kernel: a grid sized to the GPU takes groups from a work queue (a
// device counter, zero before the launch) over the systems of the launch (one,
// or the instances of a batch: group.inst indexes insts).  Each CTA allocates
// its tensor memory once and processes one group at a time; the mbarriers are
// reused, their phases counted across groups.  A wait that gives up stops the
// CTA: it lets the copy or the MMAs it waited for finish (the default limit),
// raises *status, frees its tensor memory and returns.
template <typename E>
__global__ void __launch_bounds__(256, 1) direct_tc_kernel(const TcInst* __restrict__ insts,
                                                           const PairTask* __restrict__ tasks,
                                                           const TcGroup* __restrict__ groups, int64_t ngroups,
                                                           unsigned long long* counter, float2* X, int* status,
                                                           long spin) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t mbar[3];
    __shared__ uint32_t slot;
    __shared__ long long s_g;
    __shared__ __align__(16) TcInst sI;
    __shared__ unsigned s_max;      // block maximum of an operand (float bits)
    __shared__ int s_erho[kMaxG];   // scale exponent of each pair's densities
    // TMEM: T_r in columns [0, NB), T_i in [NB, 2 NB), K^d of pair p in [2 NB + NR p, 2 NB + NR (p + 1))
    constexpr uint32_t kCols = kTmemCols;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;

    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init(&mbar[2], 1);
    }
    if (warp == 0) tc::tmem_alloc(&slot, kCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = slot;
    uint32_t ph01 = 0;   // completed phases of mbar[0] and mbar[1] (one per group)
    uint32_t ph2 = 0;    // completed phases of mbar[2] (one per pair)
    bool ok = true;

    for (;;) {
        if (tid == 0) s_g = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long gi = s_g;
        if (gi >= ngroups) break;
        const TcGroup grp = groups[gi];
        {   // the group's system
            const unsigned long long* src = (const unsigned long long*)(insts + grp.inst);
            unsigned long long* dst = (unsigned long long*)&sI;
            for (int i = tid; i < (int)(sizeof(TcInst) / 8); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        const DevSys& S = sI.S;
        const float2* __restrict__ coef = sI.coef;
        const E* __restrict__ wemb = (const E*)sI.wemb;
        const int* __restrict__ wexp = sI.wexp;
        const int ngp = sI.ngp, kg = sI.kg;
        const int nv = S.nv, nc = S.nc, nb = S.nb, P = nc * nc + nv * nv, ncc = nc * nc, nvv = nv * nv;
        const TcPlan pl = tc_plan(kg, ngp, nb, nv, nc, S.npw_max, S.ng_max);
        const int K2 = 2 * ngp;                             // K of MMA2
        const int NR = tc_rows(nv);                         // rows per pair (N of MMA2)
        const int NB = NR * kg;                             // N of MMA1 (rows of B1 and B2)
        unsigned char* Am = smem;   // the pair-density staging, then W planes, A2 (hi | lo) and the epilogue staging
        unsigned char* Bm = Am + pl.a;                      // B1 planes, then B2 (hi | lo)
        float2* RC = (float2*)(Bm + pl.b);                  // [kg][ncc][ngp] rho_cc'
        float2* ckT = (float2*)Am;
        float2* ckpT = (float2*)((unsigned char*)ckT + pl.st_coef);
        int* cnt = (int*)((unsigned char*)ckpT + pl.st_coef);
        int* list = (int*)((unsigned char*)cnt + pl.st_cnt);
        float2* rho = (float2*)((unsigned char*)list + pl.st_list);   // [ng][P]
        const size_t wpl = (size_t)128 * ngp * 2;           // one W plane (bytes)
        const size_t bpl = (size_t)NB * ngp * 2;            // one B1 plane
        const size_t a2h = (size_t)128 * K2 * 2;            // A2 hi (lo follows)
        const size_t b2h = (size_t)NB * K2 * 2;             // B2 hi (lo follows)
        const int q = grp.q, ng = S.ng[q];

        // zero the B1 planes (rows of absent pairs and of vv' >= nv^2 must be finite: they feed the scale of T)
        for (size_t e = tid * 16; e < pl.b; e += blockDim.x * 16) *(uint4*)(Bm + e) = make_uint4(0, 0, 0, 0);
        __syncthreads();

        // ---- pair densities (CUDA cores, FP32) for every pair of the group ----
        for (int p = 0; p < grp.count; ++p) {
            const PairTask t = tasks[grp.first + p];
            if (tid == 0) s_max = 0u;
            int fold[3];
            const int n3[3] = {S.n1, S.n2, S.n3};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int ik = S.kidx[3 * t.k + a], ikp = S.kidx[3 * t.kp + a];
                int iq = (ik - ikp + n3[a]) % n3[a];
                fold[a] = (ikp + iq - ik) / n3[a];
            }
            const int npkp = S.npw[t.kp];
            for (int e = tid; e < nb * S.npw_max; e += blockDim.x) {
                int b = e / S.npw_max, i = e % S.npw_max;
                ckT[i * nb + b] = coef[((int64_t)t.k * nb + b) * S.npw_max + i];
                ckpT[i * nb + b] = coef[((int64_t)t.kp * nb + b) * S.npw_max + i];
            }
            const int* gq = S.gq + (int64_t)q * S.ng_max * 3;
            const int* gk = S.gk + (int64_t)t.kp * S.npw_max * 3;
            for (int g = warp; g < ng; g += nwarp) {
                int c = 0;
                for (int j0 = 0; j0 < npkp; j0 += 32) {
                    int j = j0 + lane, idx = -1;
                    if (j < npkp) {
                        int x0 = gk[3 * j] + gq[3 * g] + fold[0] - S.blo[0];
                        int x1 = gk[3 * j + 1] + gq[3 * g + 1] + fold[1] - S.blo[1];
                        int x2 = gk[3 * j + 2] + gq[3 * g + 2] + fold[2] - S.blo[2];
                        if ((unsigned)x0 < (unsigned)S.bdim[0] && (unsigned)x1 < (unsigned)S.bdim[1] &&
                            (unsigned)x2 < (unsigned)S.bdim[2])
                            idx = S.box[(int64_t)t.k * S.bvol + ((int64_t)x0 * S.bdim[1] + x1) * S.bdim[2] + x2];
                    }
                    unsigned m = __ballot_sync(0xffffffffu, idx >= 0);
                    if (idx >= 0) list[g * S.npw_max + c + __popc(m & ((1u << lane) - 1u))] = idx | (j << 16);
                    c += __popc(m);
                }
                if (lane == 0) cnt[g] = c;
            }
            __syncthreads();
            // lanes over band pairs, up to kSlots per lane in one pass over the overlap list
            // (independent accumulators: cc' first, then vv')
            int na[kSlots], nbp[kSlots];
#pragma unroll
            for (int sl = 0; sl < kSlots; ++sl) {
                const int pp = lane + 32 * sl;
                if (pp < ncc) {
                    na[sl] = nv + pp / nc;
                    nbp[sl] = nv + pp % nc;
                } else if (pp < P) {
                    na[sl] = (pp - ncc) / nv;
                    nbp[sl] = (pp - ncc) % nv;
                } else {
                    na[sl] = nbp[sl] = -1;
                }
            }
            for (int g = warp; g < ng; g += nwarp) {
                const int* L = list + g * S.npw_max;
                const int len = cnt[g];
                float2 acc[kSlots];
#pragma unroll
                for (int sl = 0; sl < kSlots; ++sl) acc[sl] = make_float2(0.f, 0.f);
                // four list entries per iteration, their loads issued before the arithmetic
                int e = 0;
                for (; e + 3 < len; e += 4) {
                    const int4 ij = make_int4(L[e], L[e + 1], L[e + 2], L[e + 3]);   // L is 4-byte aligned only
                    const float2* a0 = ckT + (ij.x & 0xffff) * nb;
                    const float2* b0 = ckpT + (ij.x >> 16) * nb;
                    const float2* a1 = ckT + (ij.y & 0xffff) * nb;
                    const float2* b1 = ckpT + (ij.y >> 16) * nb;
                    const float2* a2 = ckT + (ij.z & 0xffff) * nb;
                    const float2* b2 = ckpT + (ij.z >> 16) * nb;
                    const float2* a3 = ckT + (ij.w & 0xffff) * nb;
                    const float2* b3 = ckpT + (ij.w >> 16) * nb;
#pragma unroll
                    for (int sl = 0; sl < kSlots; ++sl)
                        if (na[sl] >= 0) {
                            const float2 x0 = a0[na[sl]], y0 = b0[nbp[sl]], x1 = a1[na[sl]], y1 = b1[nbp[sl]];
                            const float2 x2 = a2[na[sl]], y2 = b2[nbp[sl]], x3 = a3[na[sl]], y3 = b3[nbp[sl]];
                            cmacc32(acc[sl], x0, y0);
                            cmacc32(acc[sl], x1, y1);
                            cmacc32(acc[sl], x2, y2);
                            cmacc32(acc[sl], x3, y3);
                        }
                }
                for (; e < len; ++e) {
                    const int ij = L[e];
                    const float2* a = ckT + (ij & 0xffff) * nb;
                    const float2* b = ckpT + (ij >> 16) * nb;
#pragma unroll
                    for (int sl = 0; sl < kSlots; ++sl)
                        if (na[sl] >= 0) cmacc32(acc[sl], a[na[sl]], b[nbp[sl]]);
                }
#pragma unroll
                for (int sl = 0; sl < kSlots; ++sl)
                    if (na[sl] >= 0) rho[g * P + lane + 32 * sl] = acc[sl];
            }
            __syncthreads();
            // one scale for all densities of the pair
            float mx = 0.f;
            for (int e = tid; e < ng * P; e += blockDim.x) mx = fmaxf(mx, fmaxf(fabsf(rho[e].x), fabsf(rho[e].y)));
            const int erho = scale_exp(block_max(mx, &s_max));
            const float srho = pow2f(erho);
            if (tid == 0) s_erho[p] = erho;
            // B1 rows p*NR + vv': planes rho_r, rho_i, -rho_i of rho_vv' (hi, lo), K index Q; rho_cc' kept for MMA2
            for (int e = tid; e < nvv * ngp; e += blockDim.x) {
                const int vv = e / ngp, Q = e % ngp;
                const float2 r = Q < ng ? rho[Q * P + ncc + vv] : make_float2(0.f, 0.f);
                const uint32_t o = core_off(p * NR + vv, Q, ngp);
                E h, l;
                split16(r.x * srho, h, l);
                *(E*)(Bm + o) = h;
                *(E*)(Bm + bpl + o) = l;
                split16(r.y * srho, h, l);
                *(E*)(Bm + 2 * bpl + o) = h;
                *(E*)(Bm + 3 * bpl + o) = l;
                split16(-r.y * srho, h, l);
                *(E*)(Bm + 4 * bpl + o) = h;
                *(E*)(Bm + 5 * bpl + o) = l;
            }
            for (int e = tid; e < ncc * ngp; e += blockDim.x) {
                const int cc = e / ngp, Q = e % ngp;
                RC[((size_t)p * ncc + cc) * ngp + Q] = Q < ng ? rho[Q * P + cc] : make_float2(0.f, 0.f);
            }
            __syncthreads();
        }

        // ---- W(q) into the region of the staging, now dead (generic-proxy accesses ordered before the bulk copy) ----
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)(4 * wpl);
            tc::mbar_expect_tx(&mbar[0], bytes);
            tc::bulk_g2s(Am, wemb + (size_t)q * 4 * 128 * ngp, bytes, &mbar[0]);
            s_max = 0u;   // read only after the barriers below
        }
        // ---- MMA1: T_r and T_i for all pairs (M = 128, N = NR kg, K = ngp) ----
        // a wait that gives up still lets the operation it waited for finish (the
        // default limit) before the region is reused, TMEM is freed or the CTA exits
        const bool got_w = tc::mbar_wait(&mbar[0], ph01 & 1u, spin);
        if (!got_w) tc::mbar_wait(&mbar[0], ph01 & 1u, kMbarSpinLimit);
        ok = __syncthreads_and(got_w) != 0;
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        const uint32_t idesc1 = tc::idesc_f16(128, NB, Elem<E>::kBf16);
        if (tid == 0 && ok) {
            const uint32_t lbo = 128, sbo = (uint32_t)(ngp / 8) * 128;
            const uint32_t a0 = tc::smem_u32(Am), b0 = tc::smem_u32(Bm);
            const uint32_t Wr = a0, Wi = a0 + 2 * (uint32_t)wpl;
            const uint32_t Rr = b0, Ri = b0 + 2 * (uint32_t)bpl, Rn = b0 + 4 * (uint32_t)bpl;
            // d += A B over the three split products (A_hi B_hi, A_hi B_lo, A_lo B_hi)
            auto chain = [&](uint32_t d, uint32_t A, uint32_t B, bool first) {
                for (int prod = 0; prod < 3; ++prod) {
                    const uint32_t ab = A + (prod == 2 ? (uint32_t)wpl : 0u);
                    const uint32_t bb = B + (prod == 1 ? (uint32_t)bpl : 0u);
                    for (int ks = 0; ks < ngp / 16; ++ks)
                        tc::mma_f16(d, tc::smem_desc(ab + ks * 256, lbo, sbo), tc::smem_desc(bb + ks * 256, lbo, sbo),
                                    idesc1, !(first && prod == 0 && ks == 0));
                }
            };
            chain(tmem, Wr, Rr, true);                    // T_r = Wr rho_r + Wi rho_i
            chain(tmem, Wi, Ri, false);
            chain(tmem + (uint32_t)NB, Wi, Rr, true);     // T_i = Wi rho_r - Wr rho_i
            chain(tmem + (uint32_t)NB, Wr, Rn, false);
            tc::mma_commit(&mbar[1]);
        }
        if (ok) {
            const bool got = tc::mbar_wait(&mbar[1], ph01 & 1u, spin);
            if (!got) tc::mbar_wait(&mbar[1], ph01 & 1u, kMbarSpinLimit);
            ok = __syncthreads_and(got) != 0;
        }
        ++ph01;
        tc::fence_after();
        // ---- T: TMEM -> scale -> split -> B2 (rows p*NR + vv'; K index Q for T_r, ngp + Q for T_i) ----
        int eT = 0;
        if (ok) {
            const int row = 32 * (warp & 3) + lane;                 // lane of TMEM = Q
            const int half = warp >> 2;                             // warps 0..3: T_r, 4..7: T_i
            const uint32_t tbase = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(half * NB);
            float mx = 0.f;
            for (int cb = 0; cb < NB; cb += 8) {
                float v[8];
                tc::tmem_ld8(tbase + (uint32_t)cb, v);
                if (row < ngp)
#pragma unroll
                    for (int j = 0; j < 8; ++j) mx = fmaxf(mx, fabsf(v[j]));
            }
            eT = scale_exp(block_max(mx, &s_max));
            const float sT = pow2f(eT);
            for (int cb = 0; cb < NB; cb += 8) {
                float v[8];
                tc::tmem_ld8(tbase + (uint32_t)cb, v);
                if (row < ngp) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const uint32_t o = core_off(cb + j, half * ngp + row, K2);
                        E h, l;
                        split16(v[j] * sT, h, l);
                        *(E*)(Bm + o) = h;
                        *(E*)(Bm + b2h + o) = l;
                    }
                }
            }
        }
        // ---- MMA2 per pair: K^d = rho_cc'^T T (M = 128, N = NR, K = 2 ngp) ----
        const uint32_t idesc2 = tc::idesc_f16(128, NR, Elem<E>::kBf16);
        for (int p = 0; p < grp.count && ok; ++p) {
            const float2* rc = RC + (size_t)p * ncc * ngp;
            const float srho = pow2f(s_erho[p]);
            for (int e = tid; e < 128 * ngp; e += blockDim.x) {
                const int m = e / ngp, Q = e % ngp;
                float re = 0.f, re2 = 0.f;   // values at k = Q and k = ngp + Q
                if (m < ncc) {
                    float2 r = rc[m * ngp + Q];
                    re = r.x;
                    re2 = -r.y;
                } else if (m < 2 * ncc) {
                    float2 r = rc[(m - ncc) * ngp + Q];
                    re = r.y;
                    re2 = r.x;
                }
                E h, l;
                split16(re * srho, h, l);
                *(E*)(Am + core_off(m, Q, K2)) = h;
                *(E*)(Am + a2h + core_off(m, Q, K2)) = l;
                split16(re2 * srho, h, l);
                *(E*)(Am + core_off(m, ngp + Q, K2)) = h;
                *(E*)(Am + a2h + core_off(m, ngp + Q, K2)) = l;
            }
            tc::fence_proxy_async();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (tid == 0) {
                const uint32_t lbo = 128, sbo = (uint32_t)(K2 / 8) * 128;
                const uint32_t a0 = tc::smem_u32(Am), b0 = tc::smem_u32(Bm) + (uint32_t)core_off(p * NR, 0, K2);
                const uint32_t d = tmem + 2 * (uint32_t)NB + (uint32_t)(NR * p);
                for (int prod = 0; prod < 3; ++prod) {
                    const uint32_t ab = a0 + (prod == 2 ? (uint32_t)a2h : 0u);
                    const uint32_t bb = b0 + (prod == 1 ? (uint32_t)b2h : 0u);
                    for (int ks = 0; ks < K2 / 16; ++ks)
                        tc::mma_f16(d, tc::smem_desc(ab + ks * 256, lbo, sbo), tc::smem_desc(bb + ks * 256, lbo, sbo),
                                    idesc2, (prod | ks) != 0);
                }
                tc::mma_commit(&mbar[2]);
            }
            const bool got = tc::mbar_wait(&mbar[2], ph2 & 1u, spin);
            if (!got) tc::mbar_wait(&mbar[2], ph2 & 1u, kMbarSpinLimit);
            ++ph2;
            ok = __syncthreads_and(got) != 0;
            tc::fence_after();
        }
        // ---- epilogue: TMEM -> staging (A region) -> -K^d / V into the tile ----
        float* EPI = (float*)Am;   // [kg][NR][128]
        if (ok && warp < 4) {
            const int row = 32 * warp + lane;
            for (int p = 0; p < grp.count; ++p)
                for (int cb = 0; cb < NR; cb += 8) {
                    float v[8];
                    tc::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(2 * NB + NR * p + cb), v);
#pragma unroll
                    for (int j = 0; j < 8; ++j) EPI[((size_t)p * NR + cb + j) * 128 + row] = v[j];
                }
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (ok) {
            const int B = nv * nc;
            for (int p = 0; p < grp.count; ++p) {
                const PairTask t = tasks[grp.first + p];
                // K^d = acc / (2^eW 2^(2 erho) 2^eT) and the factor -1/V
                const float scale = ldexpf((float)(-S.inv_vol), -(wexp[q] + 2 * s_erho[p] + eT));
                float2* Xt = X + t.xoff;
                for (int e = tid; e < B * B; e += blockDim.x) {
                    const int r = e % B, col = e / B;
                    const int v = r / nc, c = r % nc, vp = col / nc, cp = col % nc;
                    const float* ep = EPI + ((size_t)p * NR + v * nv + vp) * 128;
                    float2 val = make_float2(scale * ep[c * nc + cp], scale * ep[ncc + c * nc + cp]);
                    Xt[(int64_t)(t.col0 + col) * t.ld + t.row0 + r] = val;
                    if (t.flags & 1) Xt[(int64_t)(t.row0 + r) * t.ld + t.col0 + col] = make_float2(val.x, -val.y);
                }
            }
        }
        if (!ok) break;      // uniform: ok comes from __syncthreads_and
        __syncthreads();     // shared memory, s_g and sI are reused by the next group
    }
    if (!ok && tid == 0) atomicExch(status, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// per q: the exponent that brings max |Re W|, |Im W| (head and wings dropped at q = 0) to [2^13, 2^14)
__global__ void wexp_kernel(DevSys S, int* wexp) {
    __shared__ unsigned s_max;
    const int q = blockIdx.x, ng = S.ng[q];
    if (threadIdx.x == 0) s_max = 0u;
    __syncthreads();
    float mx = 0.f;
    for (int e = threadIdx.x; e < ng * ng; e += blockDim.x) {
        const int Q = e / ng, Qp = e % ng;
        if (q == 0 && (Q == S.g0 || Qp == S.g0)) continue;
        const double2 w = S.w[((int64_t)q * S.ng_max + Q) * S.ng_max + Qp];
        mx = fmaxf(mx, (float)fmax(fabs(w.x), fabs(w.y)));
    }
    const int e = scale_exp(block_max(mx, &s_max));
    if (threadIdx.x == 0) wexp[q] = e;
}

// W(q) 2^wexp[q] as four planes in the core-matrix layout (128 rows Q x ngp
// columns Q' each): Wr hi, Wr lo, Wi hi, Wi lo; zero padded; at q = 0 the
// head and wings are dropped.
template <typename E>
__global__ void wemb_kernel(DevSys S, int ngp, const int* __restrict__ wexp, E* out) {
    const int64_t per = (int64_t)128 * ngp;
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)S.nk * 2 * per) return;
    const int q = (int)(id / (2 * per));
    const int part = (int)((id / per) % 2);   // 0: Re W, 1: Im W
    const int m = (int)((id % per) / ngp), k = (int)(id % ngp);
    const int ng = S.ng[q];
    float v = 0.f;
    if (m < ng && k < ng && !(q == 0 && (m == S.g0 || k == S.g0))) {
        const double2 w = S.w[((int64_t)q * S.ng_max + m) * S.ng_max + k];
        v = (float)ldexp(part == 0 ? w.x : w.y, wexp[q]);
    }
    E h, l;
    split16(v, h, l);
    unsigned char* base = (unsigned char*)(out + (int64_t)q * 4 * per + (int64_t)(2 * part) * per);
    *(E*)(base + core_off(m, k, ngp)) = h;
    *(E*)(base + per * sizeof(E) + core_off(m, k, ngp)) = l;
}

int tc_supported(const DevSys& s, int& ngp, size_t& smem, int* kg_out) {
    ngp = (s.ng_max + 15) / 16 * 16;
    if (ngp > 128) return fail(BSE_EUNSUPPORTED, "split precision needs NG <= 128 (have %d)", s.ng_max);
    if (3 * tc_rows(s.nv) > kTmemCols) return fail(BSE_EUNSUPPORTED, "split precision needs nv <= 8");
    if (2 * s.nc * s.nc > 128) return fail(BSE_EUNSUPPORTED, "split precision needs nc <= 8");
    if (s.npw_max > 65535) return fail(BSE_EUNSUPPORTED, "npw_max > 65535");
    smem = 0;
    for (int kg = kMaxG; kg >= 1; kg /= 2) {
        if (3 * tc_rows(s.nv) * kg > kTmemCols) continue;
        smem = tc_plan(kg, ngp, s.nb, s.nv, s.nc, s.npw_max, s.ng_max).total;
        if (smem <= kSmemBudget) {
            smem = zmax(smem, kSmemFloor);
            if (kg_out) *kg_out = kg;
            return BSE_OK;
        }
    }
    return fail(BSE_EUNSUPPORTED, "split precision needs %zu bytes of shared memory", smem);
}

int launch_wemb(const DevSys& s, int ngp, int fp16, void* out, int* wexp, cudaStream_t st) {
    wexp_kernel<<<(unsigned)s.nk, 256, 0, st>>>(s, wexp);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BSE_ECUDA, "wexp launch: %s", cudaGetErrorString(e));
    int64_t n = (int64_t)s.nk * 2 * 128 * ngp;   // one thread per (q, Re/Im, row, column)
    if (fp16)
        wemb_kernel<__half><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, ngp, wexp, (__half*)out);
    else
        wemb_kernel<__nv_bfloat16><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, ngp, wexp, (__nv_bfloat16*)out);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BSE_ECUDA, "wemb launch: %s", cudaGetErrorString(e));
    return BSE_OK;
}

// dynamic shared memory of a system's plan with kg pairs per group (0 if it does not fit)
size_t tc_smem(const DevSys& s, int ngp, int kg) {
    if (3 * tc_rows(s.nv) * kg > kTmemCols) return 0;
    const size_t sm = tc_plan(kg, ngp, s.nb, s.nv, s.nc, s.npw_max, s.ng_max).total;
    return sm <= kSmemBudget ? zmax(sm, kSmemFloor) : 0;
}

template <typename E>
static int launch_direct_tc_t(const TcInst* insts, size_t smem, const PairTask* tasks, const TcGroup* groups,
                              int64_t ngroups, unsigned long long* counter, void* X, int* status, cudaStream_t st,
                              long wait_polls) {
    cudaError_t e = cudaFuncSetAttribute(direct_tc_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct_tc smem %zu: %s", smem, cudaGetErrorString(e));
    // the whole carveout as shared memory, so that two CTAs share an SM when their plans fit
    e = cudaFuncSetAttribute(direct_tc_kernel<E>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct_tc carveout: %s", cudaGetErrorString(e));
    int dev = 0, sms = 0, per_sm = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_tc_kernel<E>, 256, smem));
    if (per_sm < 1) return fail(BSE_EUNSUPPORTED, "tensor-core kernel: no CTA fits an SM");
    per_sm = per_sm > 2 ? 2 : per_sm;   // 2 x 256 TMEM columns per SM
    const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, ngroups);
    direct_tc_kernel<E><<<(unsigned)grid, 256, smem, st>>>(insts, tasks, groups, ngroups, counter, (float2*)X, status,
                                                           wait_limit(wait_polls, kMbarSpinLimit));
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct_tc launch: %s", cudaGetErrorString(e));
    return BSE_OK;
}

int launch_direct_tc(const TcInst* insts, int fp16, size_t smem, const PairTask* tasks, const TcGroup* groups,
                     int64_t ngroups, unsigned long long* counter, void* X, int* status, cudaStream_t st,
                     long wait_polls) {
    if (ngroups == 0) return BSE_OK;
    return fp16 ? launch_direct_tc_t<__half>(insts, smem, tasks, groups, ngroups, counter, X, status, st, wait_polls)
                : launch_direct_tc_t<__nv_bfloat16>(insts, smem, tasks, groups, ngroups, counter, X, status, st,
                                                    wait_polls);
}

}  // namespace bse
