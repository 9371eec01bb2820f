// Direct term of the electron-hole Hamiltonian, one k pair per CTA, on CUDA
// cores, in FP64 or FP32 (template over the real type R):
//
//   rho_nn'(k,k';Q) = sum_{p' in S_k'} conj(c_kn(p' + Q)) c_k'n'(p')     (Eq. w_interaction)
//   T_vv'(Q)        = sum_Q' W_QQ'(q) conj(rho_vv'(Q'))
//   K^d[(v,c),(v',c')] = 1/V sum_Q rho_cc'(Q) T_vv'(Q)                    (Eq. BSE-eigval)
//
// written as -K^d into a column-major tile (the diagonal eps_c - eps_v - W^div
// is added in FP64 by the projection).  At q = 0 the head and wings of W are
// dropped (Sec. III.B).
//
// The pair densities use compacted overlap lists: for each Q the plane waves
// p' with p' + Q in S_k are gathered once (warp ballot), and a warp sweeps a
// list.  In FP32 a lane takes a 4 x 4 tile of band pairs and a group of list
// entries (8 coefficients from shared memory per 16 complex multiply-adds; the
// groups summed by shuffles); in FP64, where the FP64 pipe bounds the loop, a
// lane takes up to four band pairs and every entry.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace bse {

template <typename R>
struct C2;
template <>
struct C2<double> {
    using T = double2;
};
template <>
struct C2<float> {
    using T = float2;
};

template <typename V>
__device__ __forceinline__ void cmac(V& acc, V a, V b) {   // acc += a * b
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <typename V>
__device__ __forceinline__ void cmacc(V& acc, V a, V b) {  // acc += conj(a) * b
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// shared-memory plan of one CTA
struct DirectPlan {
    size_t coef, cnt, list, stage, rho, T, total;
};

__host__ __device__ inline DirectPlan direct_plan(int cplx_bytes, int nb, int nv, int nc, int npw_max, int ng_max) {
    DirectPlan p;
    p.coef = al16((size_t)cplx_bytes * npw_max * nb);                 // one k
    p.cnt = al16(sizeof(int) * (size_t)ng_max);
    p.list = al16(sizeof(int) * (size_t)ng_max * npw_max);
    p.stage = 2 * p.coef + p.cnt + p.list;
    p.T = al16((size_t)cplx_bytes * ng_max * nv * nv);
    p.rho = al16((size_t)cplx_bytes * ng_max * (nc * nc + nv * nv));
    size_t region = p.stage > p.T ? p.stage : p.T;                     // T reuses the staging region
    p.total = region + p.rho;
    return p;
}


constexpr int kMaxPairs = 128;   // band pairs nc^2 + nv^2 per k pair (their 4 x 4 tiles fit one warp)
constexpr int kRhoSlots = kMaxPairs / 32;   // band pairs per lane in the FP64 pair-density loop

// One k pair (task t) of system I with the whole CTA; smem: the dynamic shared
// memory of the CTA (direct_plan of the system).
template <typename R>
__device__ __forceinline__ void direct_task(const DirectInst& I, const PairTask t, typename C2<R>::T* X,
                                            unsigned char* smem) {
    using V = typename C2<R>::T;
    const DevSys& S = I.S;
    const V* __restrict__ coef = (const V*)I.coef;
    const V* __restrict__ wq = (const V*)I.w;
    const int nv = S.nv, nc = S.nc, nb = S.nb, B = nv * nc, P = nc * nc + nv * nv;
    const DirectPlan pl = direct_plan((int)sizeof(V), nb, nv, nc, S.npw_max, S.ng_max);
    V* ckT = (V*)smem;                                      // [npw][nb] at k
    V* ckpT = (V*)(smem + pl.coef);                         // [npw][nb] at k'
    int* cnt = (int*)(smem + 2 * pl.coef);                  // [ng]
    int* list = (int*)(smem + 2 * pl.coef + pl.cnt);        // [ng][npw_max]: i | j << 16
    V* T = (V*)smem;                                        // [ng][nv*nv], after rho
    size_t region = pl.stage > pl.T ? pl.stage : pl.T;
    V* rho = (V*)(smem + region);                           // [ng][P]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;

    // q = k - k' and the fold f_k' + f_q - f_k
    int fold[3], iq[3];
    const int n[3] = {S.n1, S.n2, S.n3};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int ik = S.kidx[3 * t.k + a], ikp = S.kidx[3 * t.kp + a];
        iq[a] = (ik - ikp + n[a]) % n[a];
        fold[a] = (ikp + iq[a] - ik) / n[a];
    }
    const int q = (iq[0] * S.n2 + iq[1]) * S.n3 + iq[2];
    const int ng = S.ng[q], npk = S.npw[t.k], npkp = S.npw[t.kp];

    // stage both coefficient sets, band fastest
    for (int e = threadIdx.x; e < nb * S.npw_max; e += blockDim.x) {
        int b = e / S.npw_max, i = e % S.npw_max;
        ckT[i * nb + b] = coef[((int64_t)t.k * nb + b) * S.npw_max + i];
        ckpT[i * nb + b] = coef[((int64_t)t.kp * nb + b) * S.npw_max + i];
    }
    // compacted overlap list of each Q: (i in S_k, j in S_k') with p'_j + Q = p_i
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
    (void)npk;
    __syncthreads();

    if constexpr (sizeof(R) == 4) {
        // rho: one warp per Q.  The band pairs form an nc x nc (cc') and an nv x nv (vv') matrix,
        // cut into tiles of up to 4 x 4; lane = (entry group gid, tile tau): the lane sums its
        // tile over the list entries gid, gid + G, ... (4 + 4 coefficients loaded per entry for
        // 16 complex multiply-adds), and the G groups are summed by shuffles at the end.
        const int ntc = (nc + 3) >> 2, ntv = (nv + 3) >> 2, NT = ntc * ntc + ntv * ntv;
        const int G = 32 / NT, tau = lane % NT, gid = lane / NT;
        int ra, cb, nrow, ncol, pbase, pstride;   // tile rows / columns (band indices), output p = pbase + u pstride + w
        if (tau < ntc * ntc) {
            const int tr = tau / ntc, tc = tau % ntc;
            ra = nv + 4 * tr;
            cb = nv + 4 * tc;
            nrow = min(4, nc - 4 * tr);
            ncol = min(4, nc - 4 * tc);
            pbase = (4 * tr) * nc + 4 * tc;
            pstride = nc;
        } else {
            const int tv = tau - ntc * ntc, tr = tv / ntv, tc = tv % ntv;
            ra = 4 * tr;
            cb = 4 * tc;
            nrow = min(4, nv - 4 * tr);
            ncol = min(4, nv - 4 * tc);
            pbase = nc * nc + (4 * tr) * nv + 4 * tc;
            pstride = nv;
        }
        for (int g = warp; g < ng; g += nwarp) {
            V acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w].x = acc[u][w].y = R(0);
            const int* L = list + g * S.npw_max;
            const int len = gid < G ? cnt[g] : 0;
#pragma unroll 2
            for (int e = gid; e < len; e += G) {
                const int ij = L[e];
                const V* a = ckT + (ij & 0xffff) * nb + ra;
                const V* b = ckpT + (ij >> 16) * nb + cb;
                V x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    x[u] = u < nrow ? a[u] : V{R(0), R(0)};
                    y[u] = u < ncol ? b[u] : V{R(0), R(0)};
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w) cmacc(acc[u][w], x[u], y[w]);
            }
            // sum over the entry groups: lane tau + NT k holds group k's part
            for (int off = 1; off < G; off <<= 1) {
                const bool take = gid % (2 * off) == 0 && gid + off < G;
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const R ox = __shfl_down_sync(0xffffffffu, acc[u][w].x, off * NT);
                        const R oy = __shfl_down_sync(0xffffffffu, acc[u][w].y, off * NT);
                        if (take) {
                            acc[u][w].x += ox;
                            acc[u][w].y += oy;
                        }
                    }
            }
            if (gid == 0)
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int w = 0; w < 4; ++w)
                        if (u < nrow && w < ncol) rho[g * P + pbase + u * pstride + w] = acc[u][w];
        }
    } else {
        // FP64: the FP64 pipe bounds the loop, so the lanes keep one band pair per slot
        // rho: one warp per Q, lanes over band pairs (cc' first, then vv')
        int na[kRhoSlots], nbp[kRhoSlots];
#pragma unroll
        for (int s = 0; s < kRhoSlots; ++s) {
            int p = lane + 32 * s;
            if (p < nc * nc) {
                na[s] = nv + p / nc;
                nbp[s] = nv + p % nc;
            } else if (p < P) {
                na[s] = (p - nc * nc) / nv;
                nbp[s] = (p - nc * nc) % nv;
            } else {
                na[s] = nbp[s] = -1;
            }
        }
        for (int g = warp; g < ng; g += nwarp) {
            V acc[kRhoSlots];
#pragma unroll
            for (int s = 0; s < kRhoSlots; ++s) acc[s].x = acc[s].y = R(0);
            const int* L = list + g * S.npw_max;
            const int len = cnt[g];
            // four list entries per iteration, their loads issued before the arithmetic
            int e = 0;
            for (; e + 3 < len; e += 4) {
                const int ij0 = L[e], ij1 = L[e + 1], ij2 = L[e + 2], ij3 = L[e + 3];
                const V* a0 = ckT + (ij0 & 0xffff) * nb;
                const V* b0 = ckpT + (ij0 >> 16) * nb;
                const V* a1 = ckT + (ij1 & 0xffff) * nb;
                const V* b1 = ckpT + (ij1 >> 16) * nb;
                const V* a2 = ckT + (ij2 & 0xffff) * nb;
                const V* b2 = ckpT + (ij2 >> 16) * nb;
                const V* a3 = ckT + (ij3 & 0xffff) * nb;
                const V* b3 = ckpT + (ij3 >> 16) * nb;
#pragma unroll
                for (int s = 0; s < kRhoSlots; ++s)
                    if (na[s] >= 0) {
                        const V x0 = a0[na[s]], y0 = b0[nbp[s]], x1 = a1[na[s]], y1 = b1[nbp[s]];
                        const V x2 = a2[na[s]], y2 = b2[nbp[s]], x3 = a3[na[s]], y3 = b3[nbp[s]];
                        cmacc(acc[s], x0, y0);
                        cmacc(acc[s], x1, y1);
                        cmacc(acc[s], x2, y2);
                        cmacc(acc[s], x3, y3);
                    }
            }
            for (; e < len; ++e) {
                const int ij = L[e];
                const V* a = ckT + (ij & 0xffff) * nb;
                const V* b = ckpT + (ij >> 16) * nb;
#pragma unroll
                for (int s = 0; s < kRhoSlots; ++s)
                    if (na[s] >= 0) cmacc(acc[s], a[na[s]], b[nbp[s]]);
            }
#pragma unroll
            for (int s = 0; s < kRhoSlots; ++s)
                if (na[s] >= 0) rho[g * P + lane + 32 * s] = acc[s];
        }
    }
    __syncthreads();

    // T[Q][vv'] = sum_Q' W_QQ'(q) conj(rho_vv'(Q')), head and wings dropped at q = 0
    const int nvv = nv * nv, skip = (q == 0) ? S.g0 : -1;
    const V* W = wq + (int64_t)q * S.ng_max * S.ng_max;
    for (int e = threadIdx.x; e < ng * nvv; e += blockDim.x) {
        const int Q = e / nvv, vv = e % nvv;
        V acc;
        acc.x = acc.y = R(0);
        if (Q != skip) {
            const V* wr = W + (int64_t)Q * S.ng_max;
            for (int Qp = 0; Qp < ng; ++Qp) {
                if (Qp == skip) continue;
                V r = rho[Qp * P + nc * nc + vv];
                r.y = -r.y;
                cmac(acc, wr[Qp], r);
            }
        }
        T[Q * nvv + vv] = acc;
    }
    __syncthreads();

    // -K^d block, rows (v, c) fastest for coalesced column-major stores
    V* Xt = X + t.xoff;
    const R scale = R(-S.inv_vol);
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
        const int r = e % B, col = e / B;
        const int v = r / nc, c = r % nc, vp = col / nc, cp = col % nc;
        V acc;
        acc.x = acc.y = R(0);
        for (int Q = 0; Q < ng; ++Q) cmac(acc, rho[Q * P + c * nc + cp], T[Q * nvv + v * nv + vp]);
        acc.x *= scale;
        acc.y *= scale;
        Xt[(int64_t)(t.col0 + col) * t.ld + t.row0 + r] = acc;
        if (t.flags & 1) {
            V m = acc;
            m.y = -m.y;
            Xt[(int64_t)(t.row0 + r) * t.ld + t.col0 + col] = m;
        }
    }
}

// one CTA per task; kBatch: the task's system comes from insts[flags >> 1]
// (copied into shared memory), otherwise every task uses the parameter `one`
template <typename R, bool kBatch>
__global__ void __launch_bounds__(256) direct_kernel(const DirectInst* __restrict__ insts,
                                                     const __grid_constant__ DirectInst one,
                                                     const PairTask* __restrict__ tasks, typename C2<R>::T* X) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DirectInst sI;
    const PairTask t = tasks[blockIdx.x];
    if (kBatch) {   // the task's system, copied cooperatively (one round trip)
        const unsigned long long* src = (const unsigned long long*)(insts + (t.flags >> 1));
        unsigned long long* dst = (unsigned long long*)&sI;
        for (int i = threadIdx.x; i < (int)(sizeof(DirectInst) / 8); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    direct_task<R>(kBatch ? sI : one, t, X, smem);
}

// Persistent form for batches: a grid sized to the GPU takes the tasks of all
// systems from one work queue (a device counter, zero on entry), each CTA a
// task at a time, in the order of the list (largest systems first).
template <typename R>
__global__ void __launch_bounds__(256) direct_persistent_kernel(const DirectInst* __restrict__ insts,
                                                                const PairTask* __restrict__ tasks, int64_t ntasks,
                                                                unsigned long long* counter, typename C2<R>::T* X) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DirectInst sI;
    __shared__ long long s_t;
    __shared__ int s_inst;
    if (threadIdx.x == 0) s_inst = -1;
    for (;;) {
        if (threadIdx.x == 0) s_t = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long ti = s_t;
        if (ti >= ntasks) break;
        const PairTask t = tasks[ti];
        const int inst = t.flags >> 1;
        if (inst != s_inst) {   // uniform: every thread reads the same s_inst
            const unsigned long long* src = (const unsigned long long*)(insts + inst);
            unsigned long long* dst = (unsigned long long*)&sI;
            for (int i = threadIdx.x; i < (int)(sizeof(DirectInst) / 8); i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) s_inst = inst;
        }
        direct_task<R>(sI, t, X, smem);
        __syncthreads();   // shared memory and s_t are reused by the next task
    }
}

template <typename R, bool kBatch>
static int launch_direct_t(const DirectInst* insts, const DirectInst& one, const DevSys& s, const PairTask* tasks,
                           int64_t ntasks, void* X, cudaStream_t st) {
    using V = typename C2<R>::T;
    if (ntasks == 0) return BSE_OK;
    if (s.nc * s.nc + s.nv * s.nv > kMaxPairs)
        return fail(BSE_EUNSUPPORTED, "nc^2 + nv^2 > %d is not supported", kMaxPairs);
    if (s.npw_max > 65535) return fail(BSE_EUNSUPPORTED, "npw_max > 65535");
    DirectPlan pl = direct_plan((int)sizeof(V), s.nb, s.nv, s.nc, s.npw_max, s.ng_max);
    if (pl.total + sizeof(DirectInst) > 227 * 1024)
        return fail(BSE_EUNSUPPORTED, "direct kernel needs %zu bytes of shared memory", pl.total);
    cudaError_t e = cudaFuncSetAttribute(direct_kernel<R, kBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pl.total);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct smem %zu: %s", pl.total, cudaGetErrorString(e));
    // the whole carveout as shared memory: as many CTAs per SM as their plans allow
    e = cudaFuncSetAttribute(direct_kernel<R, kBatch>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct carveout: %s", cudaGetErrorString(e));
    for (int64_t off = 0; off < ntasks; off += 1 << 30) {
        int64_t nt = ntasks - off < (1 << 30) ? ntasks - off : (1 << 30);
        direct_kernel<R, kBatch><<<(unsigned)nt, 256, pl.total, st>>>(insts, one, tasks + off, (V*)X);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(BSE_ECUDA, "direct launch: %s", cudaGetErrorString(e));
    }
    return BSE_OK;
}


template <typename R>
static int launch_direct_persistent_t(const DirectInst* insts, const DevSys& s, const PairTask* tasks, int64_t ntasks,
                                      unsigned long long* counter, int threads, int ctas_per_sm, void* X,
                                      cudaStream_t st) {
    using V = typename C2<R>::T;
    if (ntasks == 0) return BSE_OK;
    if (s.nc * s.nc + s.nv * s.nv > kMaxPairs)
        return fail(BSE_EUNSUPPORTED, "nc^2 + nv^2 > %d is not supported", kMaxPairs);
    if (s.npw_max > 65535) return fail(BSE_EUNSUPPORTED, "npw_max > 65535");
    if (threads != 128 && threads != 256) return fail(BSE_EINVAL, "threads per CTA must be 128 or 256");
    DirectPlan pl = direct_plan((int)sizeof(V), s.nb, s.nv, s.nc, s.npw_max, s.ng_max);
    if (pl.total + sizeof(DirectInst) > 227 * 1024)
        return fail(BSE_EUNSUPPORTED, "direct kernel needs %zu bytes of shared memory", pl.total);
    cudaError_t e = cudaFuncSetAttribute(direct_persistent_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pl.total);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct smem %zu: %s", pl.total, cudaGetErrorString(e));
    e = cudaFuncSetAttribute(direct_persistent_kernel<R>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct carveout: %s", cudaGetErrorString(e));
    int dev = 0, sms = 0, per_sm = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, direct_persistent_kernel<R>, threads, pl.total));
    if (per_sm < 1) return fail(BSE_EUNSUPPORTED, "direct kernel: no CTA fits an SM");
    if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
    const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, ntasks);
    direct_persistent_kernel<R><<<(unsigned)grid, threads, pl.total, st>>>(insts, tasks, ntasks, counter, (V*)X);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BSE_ECUDA, "direct launch: %s", cudaGetErrorString(e));
    return BSE_OK;
}

int launch_direct_persistent(const DirectInst* insts, const DevSys& smax, int prec32, const PairTask* tasks,
                             int64_t ntasks, unsigned long long* counter, int threads, int ctas_per_sm, void* X,
                             cudaStream_t st) {
    return prec32 ? launch_direct_persistent_t<float>(insts, smax, tasks, ntasks, counter, threads, ctas_per_sm, X, st)
                  : launch_direct_persistent_t<double>(insts, smax, tasks, ntasks, counter, threads, ctas_per_sm, X,
                                                       st);
}

int launch_direct(const DirectInst& one, int prec32, const PairTask* tasks, int64_t ntasks, void* X, cudaStream_t st) {
    return prec32 ? launch_direct_t<float, false>(nullptr, one, one.S, tasks, ntasks, X, st)
                  : launch_direct_t<double, false>(nullptr, one, one.S, tasks, ntasks, X, st);
}

size_t direct_smem(const DevSys& s, int prec32) {
    return direct_plan(prec32 ? 8 : 16, s.nb, s.nv, s.nc, s.npw_max, s.ng_max).total;
}

// FP32 copies of the coefficients and of W (made once per context)
__global__ void narrow_kernel(const double2* __restrict__ in, float2* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

int launch_narrow(const double2* in, float2* out, int64_t n, cudaStream_t st) {
    if (n == 0) return BSE_OK;
    narrow_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, out, n);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BSE_ECUDA, "narrow launch: %s", cudaGetErrorString(e));
    return BSE_OK;
}

}  // namespace bse
