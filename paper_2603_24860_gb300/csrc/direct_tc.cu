// Direct term with the dense contractions on the 5th-generation tensor
// cores (tcgen05), in split precision: every operand x is stored as
// hi = bf16(x), lo = bf16(x - hi), and a product A B is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in TMEM.
//
//   rho_nn'(k,k';Q) = sum_{p'} conj(c_kn(p' + Q)) c_k'n'(p')   (CUDA cores, FP32; Eq. w_interaction)
//   T = W(q) conj(rho_vv')         MMA1, all pairs of a group share W(q)
//   K^d = 1/V rho_cc'^T T          MMA2, one pair at a time           (Eq. BSE-eigval)
//
// One CTA per group of up to kG k pairs with the same q = k - k'.  Complex
// products use real embeddings:
//   A1 = [[Wr, Wi], [Wi, -Wr]] (rows: Re T | Im T), B1 = [rho_r | rho_i]  ->  T = W conj(rho_vv')
//   A2 = [[rho_r, -rho_i], [rho_i, rho_r]] (rows: Re K | Im K), B2 = [T_r | T_i]
// W(q) (hi and lo) is prepared once per q in the core-matrix layout and
// brought in by one bulk copy that overlaps the pair densities.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_ptx.h"

namespace bse {

using tc::core_off;

constexpr int kG = 4;        // pairs per group
constexpr int kNVV = 16;     // rows of B1/B2 per pair (nv^2 padded)

struct TcPlan {
    int K;                   // 2 * NGp
    size_t a1, b, a2, rc, st_coef, st_cnt, st_list, st_rho, total;
};

__host__ __device__ inline size_t a16(size_t x) { return (x + 1023) & ~(size_t)1023; }

__host__ __device__ inline TcPlan tc_plan(int ngp, int nb, int nv, int nc, int npw_max, int ng_max) {
    TcPlan p;
    p.K = 2 * ngp;
    p.a1 = a16((size_t)2 * 128 * p.K * 2);
    p.b = a16((size_t)2 * kG * kNVV * p.K * 2);
    size_t a2 = (size_t)2 * 128 * p.K * 2, epi = (size_t)kG * kNVV * 128 * sizeof(float);
    p.a2 = a16(a2 > epi ? a2 : epi);   // also holds the epilogue staging
    p.rc = a16((size_t)kG * nc * nc * ngp * sizeof(float2));
    p.st_coef = a16((size_t)npw_max * nb * sizeof(float2));
    p.st_cnt = a16((size_t)ng_max * sizeof(int));
    p.st_list = a16((size_t)ng_max * npw_max * sizeof(int));
    p.st_rho = a16((size_t)ng_max * (nc * nc + nv * nv) * sizeof(float2));
    p.total = p.a1 + p.b + p.a2 + p.rc + 2 * p.st_coef + p.st_cnt + p.st_list + p.st_rho + 1024 + 64;
    return p;
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ void cmacc32(float2& acc, float2 a, float2 b) {   // acc += conj(a) * b
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

__global__ void __launch_bounds__(256, 1) direct_tc_kernel(DevSys S, const float2* __restrict__ coef,
                                                           const __nv_bfloat16* __restrict__ wemb,
                                                           const PairTask* __restrict__ tasks,
                                                           const TcGroup* __restrict__ groups, int ngp, float2* X,
                                                           int* status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nv = S.nv, nc = S.nc, nb = S.nb, P = nc * nc + nv * nv, ncc = nc * nc, nvv = nv * nv;
    const TcPlan pl = tc_plan(ngp, nb, nv, nc, S.npw_max, S.ng_max);
    const int K = pl.K;
    unsigned char* A1 = smem;                           // [hi | lo] 128 x K
    unsigned char* Bm = A1 + pl.a1;                     // [hi | lo] (kG*16) x K : B1, then B2
    unsigned char* A2 = Bm + pl.b;                      // [hi | lo] 128 x K
    float2* RC = (float2*)(A2 + pl.a2);                 // [kG][ncc][ngp] rho_cc'
    float2* ckT = (float2*)((unsigned char*)RC + pl.rc);
    float2* ckpT = (float2*)((unsigned char*)ckT + pl.st_coef);
    int* cnt = (int*)((unsigned char*)ckpT + pl.st_coef);
    int* list = (int*)((unsigned char*)cnt + pl.st_cnt);
    float2* rho = (float2*)((unsigned char*)list + pl.st_list);   // [ng][P]
    uint64_t* mbar = (uint64_t*)((unsigned char*)rho + pl.st_rho);
    uint32_t* slot = (uint32_t*)(mbar + 4);
    const size_t a_half = (size_t)128 * K * 2, b_half = (size_t)kG * kNVV * K * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = blockDim.x >> 5;
    const TcGroup grp = groups[blockIdx.x];
    const int q = grp.q, ng = S.ng[q];
    constexpr uint32_t kCols = 128;   // TMEM: MMA1 accumulator cols [0, 64), MMA2 [64, 128)
    constexpr long kSpin = 1l << 24;

    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init(&mbar[2], 1);
    }
    if (warp == 0) tc::tmem_alloc(slot, kCols);
    // zero B1 (its padding must be finite: A1 is zero there)
    for (size_t e = tid * 16; e < 2 * b_half; e += blockDim.x * 16) *(uint4*)(Bm + e) = make_uint4(0, 0, 0, 0);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *slot;
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)(2 * a_half);
        tc::mbar_expect_tx(&mbar[0], bytes);
        tc::bulk_g2s(A1, wemb + (size_t)q * 2 * 128 * K, bytes, &mbar[0]);
    }

    // ---- pair densities (CUDA cores, FP32) for every pair of the group ----
    for (int p = 0; p < grp.count; ++p) {
        const PairTask t = tasks[grp.first + p];
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
        for (int g = warp; g < ng; g += nwarp) {
            const int* L = list + g * S.npw_max;
            const int len = cnt[g];
            for (int p0 = 0; p0 < P; p0 += 32) {
                const int pp = p0 + lane;
                if (pp >= P) break;
                int na, nbp;
                if (pp < ncc) {
                    na = nv + pp / nc;
                    nbp = nv + pp % nc;
                } else {
                    na = (pp - ncc) / nv;
                    nbp = (pp - ncc) % nv;
                }
                float2 acc = make_float2(0.f, 0.f);
                for (int e = 0; e < len; ++e) {
                    const int ij = L[e];
                    cmacc32(acc, ckT[(ij & 0xffff) * nb + na], ckpT[(ij >> 16) * nb + nbp]);
                }
                rho[g * P + pp] = acc;
            }
        }
        __syncthreads();
        // B1 rows p*16 + vv' = [rho_r | rho_i] of rho_vv', and rho_cc' kept for MMA2
        unsigned char* B1h = Bm;
        unsigned char* B1l = Bm + b_half;
        for (int e = tid; e < nvv * ngp; e += blockDim.x) {
            const int vv = e / ngp, Q = e % ngp;
            float2 r = Q < ng ? rho[Q * P + ncc + vv] : make_float2(0.f, 0.f);
            __nv_bfloat16 h, l;
            split_bf16(r.x, h, l);
            *(__nv_bfloat16*)(B1h + core_off(p * kNVV + vv, Q, K)) = h;
            *(__nv_bfloat16*)(B1l + core_off(p * kNVV + vv, Q, K)) = l;
            split_bf16(r.y, h, l);
            *(__nv_bfloat16*)(B1h + core_off(p * kNVV + vv, ngp + Q, K)) = h;
            *(__nv_bfloat16*)(B1l + core_off(p * kNVV + vv, ngp + Q, K)) = l;
        }
        for (int e = tid; e < ncc * ngp; e += blockDim.x) {
            const int cc = e / ngp, Q = e % ngp;
            RC[((size_t)p * ncc + cc) * ngp + Q] = Q < ng ? rho[Q * P + cc] : make_float2(0.f, 0.f);
        }
        __syncthreads();
    }

    // ---- MMA1: T = W(q) conj(rho_vv') for all pairs (N = 16 * kG) ----
    bool ok = __syncthreads_and(tc::mbar_wait(&mbar[0], 0, kSpin)) != 0;
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t idesc1 = tc::idesc_f16(128, kNVV * kG, 1);
    const uint32_t lbo = 128, sbo = (uint32_t)(K / 8) * 128;
    if (tid == 0 && ok) {
        const uint32_t a0 = tc::smem_u32(A1), b0 = tc::smem_u32(Bm);
        for (int prod = 0; prod < 3; ++prod) {
            const uint32_t ab = a0 + (prod == 2 ? (uint32_t)a_half : 0u);
            const uint32_t bb = b0 + (prod == 1 ? (uint32_t)b_half : 0u);
            for (int ks = 0; ks < K / 16; ++ks)
                tc::mma_f16(tmem, tc::smem_desc(ab + ks * 256, lbo, sbo), tc::smem_desc(bb + ks * 256, lbo, sbo), idesc1,
                            (prod | ks) != 0);
        }
        tc::mma_commit(&mbar[1]);
    }
    ok = __syncthreads_and(ok && tc::mbar_wait(&mbar[1], 0, kSpin)) != 0;
    tc::fence_after();
    // ---- T: TMEM -> split -> B2 (rows p*16 + vv', K index = row of T) ----
    if (ok) {
        const int row = 32 * (warp & 3) + lane;                 // row of T = K index of B2
        const int c0 = (warp >> 2) * (kNVV * kG / 2);           // warps 4..7 take the upper columns
        for (int cb = c0; cb < c0 + kNVV * kG / 2; cb += 8) {
            float v[8];
            tc::tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cb, v);
            if (row < K) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __nv_bfloat16 h, l;
                    split_bf16(v[j], h, l);
                    *(__nv_bfloat16*)(Bm + core_off(cb + j, row, K)) = h;
                    *(__nv_bfloat16*)(Bm + b_half + core_off(cb + j, row, K)) = l;
                }
            }
        }
    }
    // ---- MMA2 per pair: K^d = rho_cc'^T T ----
    const uint32_t idesc2 = tc::idesc_f16(128, kNVV, 1);
    for (int p = 0; p < grp.count && ok; ++p) {
        const float2* rc = RC + (size_t)p * ncc * ngp;
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
            __nv_bfloat16 h, l;
            split_bf16(re, h, l);
            *(__nv_bfloat16*)(A2 + core_off(m, Q, K)) = h;
            *(__nv_bfloat16*)(A2 + a_half + core_off(m, Q, K)) = l;
            split_bf16(re2, h, l);
            *(__nv_bfloat16*)(A2 + core_off(m, ngp + Q, K)) = h;
            *(__nv_bfloat16*)(A2 + a_half + core_off(m, ngp + Q, K)) = l;
        }
        tc::fence_proxy_async();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            const uint32_t a0 = tc::smem_u32(A2), b0 = tc::smem_u32(Bm) + (uint32_t)core_off(p * kNVV, 0, K);
            const uint32_t d = tmem + 64 + 16 * p;
            for (int prod = 0; prod < 3; ++prod) {
                const uint32_t ab = a0 + (prod == 2 ? (uint32_t)a_half : 0u);
                const uint32_t bb = b0 + (prod == 1 ? (uint32_t)b_half : 0u);
                for (int ks = 0; ks < K / 16; ++ks)
                    tc::mma_f16(d, tc::smem_desc(ab + ks * 256, lbo, sbo), tc::smem_desc(bb + ks * 256, lbo, sbo),
                                idesc2, (prod | ks) != 0);
            }
            tc::mma_commit(&mbar[2]);
        }
        ok = __syncthreads_and(tc::mbar_wait(&mbar[2], (uint32_t)(p & 1), kSpin)) != 0;
        tc::fence_after();
    }
    // ---- epilogue: TMEM -> staging (A2 region) -> -K^d / V into the tile ----
    float* EPI = (float*)A2;   // [kG][16][128]
    if (ok && warp < 4) {
        const int row = 32 * warp + lane;
        for (int p = 0; p < grp.count; ++p)
            for (int cb = 0; cb < 16; cb += 8) {
                float v[8];
                tc::tmem_ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(64 + 16 * p + cb), v);
#pragma unroll
                for (int j = 0; j < 8; ++j) EPI[((size_t)p * 16 + cb + j) * 128 + row] = v[j];
            }
    }
    __syncthreads();
    if (ok) {
        const int B = nv * nc;
        const float scale = (float)(-S.inv_vol);
        for (int p = 0; p < grp.count; ++p) {
            const PairTask t = tasks[grp.first + p];
            float2* Xt = X + t.xoff;
            for (int e = tid; e < B * B; e += blockDim.x) {
                const int r = e % B, col = e / B;
                const int v = r / nc, c = r % nc, vp = col / nc, cp = col % nc;
                const float* ep = EPI + ((size_t)p * 16 + v * nv + vp) * 128;
                float2 val = make_float2(scale * ep[c * nc + cp], scale * ep[ncc + c * nc + cp]);
                Xt[(int64_t)(t.col0 + col) * t.ld + t.row0 + r] = val;
                if (t.flags & 1) Xt[(int64_t)(t.row0 + r) * t.ld + t.col0 + col] = make_float2(val.x, -val.y);
            }
        }
    }
    if (!ok && tid == 0) atomicExch(status, 1);
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// W(q) real embedding in the core-matrix layout, hi then lo, zero padded;
// at q = 0 the head and wings are dropped.
__global__ void wemb_kernel(DevSys S, int ngp, __nv_bfloat16* out) {
    const int K = 2 * ngp;
    const int64_t per = (int64_t)128 * K;
    int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)S.nk * per) return;
    const int q = (int)(id / per);
    const int m = (int)((id % per) / K), k = (int)(id % K);
    const int ng = S.ng[q];
    float v = 0.f;
    const int Q = m < ngp ? m : m - ngp, Qp = k < ngp ? k : k - ngp;
    if (m < 2 * ngp && Q < ng && Qp < ng && !(q == 0 && (Q == S.g0 || Qp == S.g0))) {
        double2 w = S.w[((int64_t)q * S.ng_max + Q) * S.ng_max + Qp];
        // [[Wr, Wi], [Wi, -Wr]]
        double x = (m < ngp) ? (k < ngp ? w.x : w.y) : (k < ngp ? w.y : -w.x);
        v = (float)x;
    }
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    __nv_bfloat16* base = out + (int64_t)q * 2 * per;
    *(__nv_bfloat16*)((unsigned char*)base + core_off(m, k, K)) = h;
    *(__nv_bfloat16*)((unsigned char*)(base + per) + core_off(m, k, K)) = l;
}

int tc_supported(const DevSys& s, int& ngp, size_t& smem) {
    ngp = (s.ng_max + 7) / 8 * 8;
    smem = tc_plan(ngp, s.nb, s.nv, s.nc, s.npw_max, s.ng_max).total;
    if (ngp > 64) return fail(BSE_EUNSUPPORTED, "split precision needs NG <= 64 (have %d)", s.ng_max);
    if (s.nv * s.nv > kNVV) return fail(BSE_EUNSUPPORTED, "split precision needs nv <= 4");
    if (2 * s.nc * s.nc > 128) return fail(BSE_EUNSUPPORTED, "split precision needs nc <= 8");
    if (s.npw_max > 65535) return fail(BSE_EUNSUPPORTED, "npw_max > 65535");
    if (smem > 227 * 1024) return fail(BSE_EUNSUPPORTED, "split precision needs %zu bytes of shared memory", smem);
    return BSE_OK;
}

int launch_wemb(const DevSys& s, int ngp, void* out, cudaStream_t st) {
    int64_t n = (int64_t)s.nk * 128 * 2 * ngp;
    wemb_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, ngp, (__nv_bfloat16*)out);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BSE_ECUDA, "wemb launch: %s", cudaGetErrorString(e));
    return BSE_OK;
}

int launch_direct_tc(const DevSys& s, const void* coef32, const void* wemb, int ngp, const PairTask* tasks,
                     const TcGroup* groups, int64_t ngroups, void* X, int* status, cudaStream_t st) {
    if (ngroups == 0) return BSE_OK;
    int ngp2;
    size_t sm;
    BSE_TRY(tc_supported(s, ngp2, sm));
    cudaError_t e = cudaFuncSetAttribute(direct_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct_tc smem %zu: %s", sm, cudaGetErrorString(e));
    for (int64_t off = 0; off < ngroups; off += 1 << 30) {
        int64_t n = ngroups - off < (1 << 30) ? ngroups - off : (1 << 30);
        direct_tc_kernel<<<(unsigned)n, 256, sm, st>>>(s, (const float2*)coef32, (const __nv_bfloat16*)wemb, tasks,
                                                      groups + off, ngp, (float2*)X, status);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(BSE_ECUDA, "direct_tc launch: %s", cudaGetErrorString(e));
    }
    return BSE_OK;
}

}  // namespace bse
