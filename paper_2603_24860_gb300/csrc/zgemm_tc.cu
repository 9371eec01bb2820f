// Z = A22 V of the two-stage reduction on the tcgen05 tensor cores (sm_103a):
// A22 = A[r1:, r1:] (m x m, double-float, Hermitian), V = [32][n] reflectors.
//
// The contraction runs over K in chunks of 64 complex columns.  In real form,
// with K' = 128 per chunk,
//   Re Z[r,l] = [Ar Ai] [Vr -Vi]^T,   Im Z[r,l] = [Ar Ai] [Vi Vr]^T,
// so the A22 chunk is one MMA operand (M = 128 rows) and the two forms of the V
// chunk are stacked as the 64 rows (N) of the other.  Within a chunk the
// operands are split exactly as in the panel update (her2k_tc.cu): a row of the
// A22 chunk and a column of the V chunk each get a power-of-two scale from their
// largest entry, are rounded to 56 bits and written as 8 balanced base-128
// digits stored pre-scaled (d_k 2^-7k, exact in bf16); the digit-pair groups
// g = k + m < 4 accumulate exactly in FP32 in TMEM, the groups 4..7 share a fifth
// accumulator.  Per chunk the five accumulators are summed in double-float,
// scaled by 2^(e_r + f_l - 14) and added to double-float accumulators held in
// registers, so the chunks combine in double-float.  CTA (row tile, split) takes
// a contiguous range of chunks; its partial Z goes to zpart[split][row][l].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dfloat.h"
#include "digits.h"
#include "grid_sync.h"
#include "internal.h"
#include "tc_ptx.h"

namespace bse {

namespace {

constexpr int kZM = 128;                                   // rows of a tile (M, TMEM lanes)
constexpr int kZL = 32;                                    // columns of Z (reflectors)
constexpr int kZN = 64;                                    // N of the MMA: [Vr -Vi] rows, then [Vi Vr] rows
constexpr int kZK = 128;                                   // K' of a chunk (64 complex columns)
constexpr int kZC = 64;                                    // complex columns per chunk
constexpr int kZDig = kDigits;
constexpr int kZExact = 4;
constexpr int kZAcc = kZExact + 1;
constexpr int kZSlots = 3;
constexpr uint32_t kZTmemCols = 512;                       // kZAcc x kZN = 320 used
constexpr size_t kZADig = (size_t)kZM * kZK * 2;           // one digit of an A22 tile chunk (32 KB)
constexpr size_t kZBDig = (size_t)kZN * kZK * 2;           // one digit of a V chunk, both forms (16 KB)
constexpr size_t kZBChunk = kZDig * kZBDig;                // 128 KB
constexpr size_t kZSmem = kZBChunk + kZSlots * kZADig + 1024;
constexpr int kZMaxSplit = 8;



// eight bf16 values (exact: pre-scaled digits) packed as one 16-byte store
__device__ __forceinline__ uint4 pack8(const float* x) {
    uint4 u;
    __nv_bfloat162 t;
    t = __floats2bfloat162_rn(x[0], x[1]);
    u.x = *reinterpret_cast<uint32_t*>(&t);
    t = __floats2bfloat162_rn(x[2], x[3]);
    u.y = *reinterpret_cast<uint32_t*>(&t);
    t = __floats2bfloat162_rn(x[4], x[5]);
    u.z = *reinterpret_cast<uint32_t*>(&t);
    t = __floats2bfloat162_rn(x[6], x[7]);
    u.w = *reinterpret_cast<uint32_t*>(&t);
    return u;
}

// A22 digits per chunk in one pass: a CTA takes 32 rows of one chunk, warp g the columns
// 8 g .. 8 g + 7 (lane = row, so the loads are coalesced over rows); the row's exponent
// per chunk (2^ex above its largest entry there) from the eight warps' maxima in shared
// memory, written for the GEMM's epilogue, then the exact digit split of the eight entries:
// the 16-byte pieces of each digit for the group's Re parts (K 8g .. 8g+7) and Im parts
// (K 64 + 8g ..), in tiles [rt][c][k] of 128 x 128 in the core-matrix layout
__global__ void __launch_bounds__(256) a22_digits_kernel(const cdf* __restrict__ A, int n, int r1, int m, int nrt,
                                                         int nch, __nv_bfloat16* Adig, int* __restrict__ ex) {
    __shared__ float s_mx[kZC / 8][32];
    const int64_t rows = (int64_t)nrt * kZM;
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5, c = blockIdx.y;
    const int r = blockIdx.x * 32 + lane;
    const int rt = r / kZM, rr = r % kZM;
    const bool live = r < m;
    const int c0 = c * kZC, cn = min(kZC, m - c0);
    const cdf* row = A + (size_t)(r1 + c0) * n + r1 + r;   // entry j of the chunk at row[j n]
    cdf z[8];
    float mx = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int j = 8 * g + u;
        z[u] = live && j < cn ? __ldcg(row + (size_t)j * n) : cdf_zero();
        mx = fmaxf(mx, fmaxf(fabsf(z[u].x), fabsf(z[u].z)));
    }
    s_mx[g][lane] = mx;
    __syncthreads();
#pragma unroll
    for (int h = 0; h < kZC / 8; ++h) mx = fmaxf(mx, s_mx[h][lane]);
    const int e = exp_above_f(mx);
    if (g == 0) ex[(size_t)c * rows + r] = e;
    float dr[8][kZDig], di[8][kZDig];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        df_digits8(z[u].x, z[u].y, e, dr[u]);
        df_digits8(z[u].z, z[u].w, e, di[u]);
    }
    unsigned char* tile = (unsigned char*)Adig + ((size_t)rt * nch + c) * kZDig * kZADig;
#pragma unroll
    for (int k = 0; k < kZDig; ++k) {
        float pr[8], pi[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            pr[u] = dr[u][k];
            pi[u] = di[u][k];
        }
        unsigned char* base = tile + (size_t)k * kZADig;
        *(uint4*)(base + tc::core_off(rr, 8 * g, kZK)) = pack8(pr);
        *(uint4*)(base + tc::core_off(rr, kZC + 8 * g, kZK)) = pack8(pi);
    }
}

// V digits: thread per (chunk c, group of 8 columns g, reflector l); the column exponent over the
// chunk; rows l of [Vr -Vi] and 32 + l of [Vi Vr] of each digit (tiles [c][k] of 64 x 128)
__global__ void v_digits_kernel(const cdf* __restrict__ V, int n, int r1, int m, int nch, __nv_bfloat16* Bdig,
                                int* fy) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nch * (kZC / 8) * kZL) return;
    const int l = gid % kZL, g = (gid / kZL) % (kZC / 8), c = gid / (kZL * (kZC / 8));
    const int c0 = c * kZC, cn = min(kZC, m - c0);
    const cdf* col = V + (size_t)l * n + r1 + c0;
    float mx = 0.f;
    for (int j = 0; j < cn; ++j) {
        const cdf z = __ldcg(col + j);
        mx = fmaxf(mx, fmaxf(fabsf(z.x), fabsf(z.z)));
    }
    const int e = exp_above_f(mx);
    if (g == 0) fy[c * kZL + l] = e;
    float dr[8][kZDig], di[8][kZDig];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int j = 8 * g + u;
        const cdf z = j < cn ? __ldcg(col + j) : cdf_zero();
        df_digits8(z.x, z.y, e, dr[u]);
        df_digits8(z.z, z.w, e, di[u]);
    }
    unsigned char* tile = (unsigned char*)Bdig + (size_t)c * kZBChunk;
#pragma unroll
    for (int k = 0; k < kZDig; ++k) {
        float pr[8], pi[8], ni[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            pr[u] = dr[u][k];
            pi[u] = di[u][k];
            ni[u] = -di[u][k];
        }
        unsigned char* base = tile + (size_t)k * kZBDig;
        *(uint4*)(base + tc::core_off(l, 8 * g, kZK)) = pack8(pr);   // [Vr -Vi]
        *(uint4*)(base + tc::core_off(l, kZC + 8 * g, kZK)) = pack8(ni);
        *(uint4*)(base + tc::core_off(kZL + l, 8 * g, kZK)) = pack8(pi);   // [Vi Vr]
        *(uint4*)(base + tc::core_off(kZL + l, kZC + 8 * g, kZK)) = pack8(pr);
    }
}

struct ZArgs {
    const __nv_bfloat16* Adig;   // [nrt][nch][8][128 x 128]
    const __nv_bfloat16* Bdig;   // [nch][8][64 x 128]
    const int* ex;               // [nch][nrt * 128] row exponents
    const int* fy;               // [nch][32] column exponents
    cdf* zpart;                  // [split][m][32]
    int m, nrt, nch, nsplit;
    int* status;
    long spin;
};

// five accumulators of one output (exact FP32 values) summed in double-float
__device__ __forceinline__ float2 zsum5(const uint32_t (&v)[kZAcc][8], int j) {
    float h, l, h2, l2;
    two_sum(__uint_as_float(v[0][j]), __uint_as_float(v[1][j]), h, l);
    two_sum(__uint_as_float(v[2][j]), __uint_as_float(v[3][j]), h2, l2);
    const float2 s = df_add(make_float2(h, l), make_float2(h2, l2));
    return df_add(s, make_float2(__uint_as_float(v[4][j]), 0.f));
}

// mbarrier wait that gives up after `limit` polls or once another role has raised the
// CTA's abort flag
__device__ __forceinline__ bool ws_wait(uint64_t* mb, uint32_t parity, long limit, volatile int* abort) {
    for (long it = 0; it < limit; ++it) {
        if (tc::mbar_wait(mb, parity, 1)) return true;
        if ((it & 15) == 15 && *abort) return false;
    }
    return false;
}

// CTA (rt = blockIdx.x, split = blockIdx.y) takes chunks [nch s / S, nch (s + 1) / S), with
// warp-specialised roles: warp 4 (one lane) copies the V chunk into its buffer once the MMAs of
// the previous chunk are done and streams the 8 digits of the A22 chunk through three slots as
// they free up; warp 5 (one lane) issues the MMAs as operands land, once the drain of the previous
// chunk has released TMEM; warps 0-3 drain each chunk's accumulators (a warp per 32 TMEM lanes =
// rows) into double-float registers.  X item j = digit j % 8 of chunk c_lo + j / 8 uses slot
// j % 3 (its copy the (j / 3)-th completion of mb_full[slot], its MMAs the (j / 3)-th commit to
// mb_empty[slot]); one completion of mb_y, mb_acc and mb_free per chunk.
constexpr int kZWThreads = 192;
__global__ void __launch_bounds__(kZWThreads, 1) zgemm_tc_kernel(ZArgs a) {
    extern __shared__ __align__(1024) unsigned char zsm_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)zsm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* Bs = smem;
    unsigned char* As = smem + kZBChunk;
    __shared__ __align__(8) uint64_t mb_y, mb_full[kZSlots], mb_empty[kZSlots], mb_acc, mb_free, mb_fin;
    __shared__ uint32_t slot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&mb_y, 1);
        tc::mbar_init(&mb_acc, 1);
        tc::mbar_init(&mb_free, 4);
        tc::mbar_init(&mb_fin, 1);
        for (int i = 0; i < kZSlots; ++i) {
            tc::mbar_init(&mb_full[i], 1);
            tc::mbar_init(&mb_empty[i], 1);
        }
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&slot, kZTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = slot;
    volatile int* abort = &s_abort;
    const int rt = blockIdx.x, sp = blockIdx.y;
    const int c_lo = (int)((int64_t)a.nch * sp / a.nsplit), c_hi = (int)((int64_t)a.nch * (sp + 1) / a.nsplit);
    const int nchunk = c_hi - c_lo;
    auto fail_now = [&]() {
        *abort = 1;
        atomicExch(a.status, 1);
    };
    if (warp == 4) {
        if (lane == 0) {   // producer
            int last[kZSlots] = {-1, -1, -1}, ys = 0;
            bool ok = true;
            for (int cl = 0; cl < nchunk && ok; ++cl) {
                if (cl > 0 && !(ok = ws_wait(&mb_acc, (uint32_t)((cl - 1) & 1), a.spin, abort))) break;
                tc::mbar_expect_tx(&mb_y, (uint32_t)kZBChunk);
                tc::bulk_g2s(Bs, (const unsigned char*)a.Bdig + (size_t)(c_lo + cl) * kZBChunk, (uint32_t)kZBChunk,
                             &mb_y);
                ++ys;
                for (int k = 0; k < kZDig; ++k) {
                    const int j = cl * kZDig + k, sl = j % kZSlots;
                    if (j >= kZSlots && !(ok = ws_wait(&mb_empty[sl], (uint32_t)(((j - kZSlots) / kZSlots) & 1),
                                                       a.spin, abort)))
                        break;
                    tc::mbar_expect_tx(&mb_full[sl], (uint32_t)kZADig);
                    tc::bulk_g2s(As + sl * kZADig,
                                 (const unsigned char*)a.Adig + (((size_t)rt * a.nch + c_lo + cl) * kZDig + k) * kZADig,
                                 (uint32_t)kZADig, &mb_full[sl]);
                    last[sl] = j;
                }
            }
            if (!ok) fail_now();
            // every copy issued has landed before the CTA may leave
            for (int sl = 0; sl < kZSlots; ++sl)
                if (last[sl] >= 0) tc::mbar_wait(&mb_full[sl], (uint32_t)((last[sl] / kZSlots) & 1), kMbarSpinLimit);
            if (ys > 0) tc::mbar_wait(&mb_y, (uint32_t)((ys - 1) & 1), kMbarSpinLimit);
        }
    } else if (warp == 5) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = tc::idesc_f16(kZM, kZN, 1);
            const uint32_t lbo = 128, sbo = (uint32_t)(kZK / 8) * 128;
            bool ok = true;
            for (int cl = 0; cl < nchunk && ok; ++cl) {
                if (!(ok = ws_wait(&mb_y, (uint32_t)(cl & 1), a.spin, abort))) break;
                if (cl > 0 && !(ok = ws_wait(&mb_free, (uint32_t)((cl - 1) & 1), a.spin, abort))) break;
                tc::fence_after();
                for (int k = 0; k < kZDig; ++k) {
                    const int j = cl * kZDig + k, sl = j % kZSlots;
                    if (!(ok = ws_wait(&mb_full[sl], (uint32_t)((j / kZSlots) & 1), a.spin, abort))) break;
                    tc::fence_after();
                    const uint64_t ad = tc::smem_desc(tc::smem_u32(As + sl * kZADig), lbo, sbo);
                    for (int mm = 0; mm + k < kZDig; ++mm) {
                        const int g = k + mm, acc = g < kZExact ? g : kZExact;
                        const bool first = k == 0 && (g < kZExact || mm == kZExact);
                        const uint64_t bd = tc::smem_desc(tc::smem_u32(Bs + mm * kZBDig), lbo, sbo);
                        const uint32_t d = tmem + (uint32_t)(acc * kZN);
#pragma unroll
                        for (int ks = 0; ks < kZK / 16; ++ks)
                            tc::mma_f16(d, ad + (uint64_t)(ks * 16), bd + (uint64_t)(ks * 16), idesc,
                                        (first && ks == 0) ? 0u : 1u);
                    }
                    tc::mma_commit(&mb_empty[sl]);
                }
                if (ok) tc::mma_commit(&mb_acc);
            }
            if (!ok) fail_now();
            // every MMA issued has completed before TMEM is released
            tc::mma_commit(&mb_fin);
            tc::mbar_wait(&mb_fin, 0u, kMbarSpinLimit);
        }
    } else {   // drain warps 0-3
        const int r = rt * kZM + warp * 32 + lane;
        const bool rlive = r < a.m;
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
        float zr[kZL][2], zi[kZL][2];   // double-float accumulators of Z[r][l]
#pragma unroll
        for (int l = 0; l < kZL; ++l) zr[l][0] = zr[l][1] = zi[l][0] = zi[l][1] = 0.f;
        bool ok = true;
        for (int cl = 0; cl < nchunk; ++cl) {
            const int c = c_lo + cl;
            if (!ws_wait(&mb_acc, (uint32_t)(cl & 1), a.spin, abort)) {
                ok = false;
                break;
            }
            tc::fence_after();
            const int er = rlive ? __ldg(a.ex + (size_t)c * a.nrt * kZM + r) : 0;
#pragma unroll
            for (int c0 = 0; c0 < kZL; c0 += 8) {
#pragma unroll
                for (int part = 0; part < 2; ++part) {   // real parts (columns c0..), then imaginary (32 + c0..)
                    uint32_t v[kZAcc][8];
#pragma unroll
                    for (int q = 0; q < kZAcc; ++q)
                        tc::tmem_ld8_async(tmem + lane_off + (uint32_t)(q * kZN + part * kZL + c0), v[q]);
#pragma unroll
                    for (int q = 0; q < kZAcc; ++q) tc::tmem_ld_wait(v[q]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float sc = ldexpf(1.f, er + __ldg(a.fy + c * kZL + c0 + j) - 14);
                        const float2 sv = zsum5(v, j);
                        float(&acc)[2] = part == 0 ? zr[c0 + j] : zi[c0 + j];
                        const float2 nv = df_add(make_float2(acc[0], acc[1]), make_float2(sv.x * sc, sv.y * sc));
                        acc[0] = nv.x;
                        acc[1] = nv.y;
                    }
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&mb_free)) : "memory");
        }
        if (!ok) fail_now();
        if (ok && rlive) {
            cdf* out = a.zpart + ((size_t)sp * a.m + r) * kZL;
#pragma unroll
            for (int l = 0; l < kZL; ++l) out[l] = make_float4(zr[l][0], zr[l][1], zi[l][0], zi[l][1]);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kZTmemCols);
}

}  // namespace

size_t zgemm_tc_bytes(int64_t n) {
    const int64_t nrt = (n + kZM - 1) / kZM, nch = (n + kZC - 1) / kZC;
    return (size_t)nrt * nch * kZDig * kZADig + (size_t)nch * kZBChunk + sizeof(int) * (size_t)(nch * (nrt * kZM + kZL)) +
           4096;
}

int zgemm_tc_splits(int64_t m, int sms) {
    const int nrt = (int)((m + kZM - 1) / kZM), nch = (int)((m + kZC - 1) / kZC);
    return std::max(1, std::min({kZMaxSplit, nch, (sms + nrt - 1) / nrt}));
}

int launch_zgemm_tc(const cdf* A, int64_t n64, int r1, int m, const cdf* V, void* scratch, cdf* zpart, int nsplit,
                    int* status, cudaStream_t st, long wait_polls) {
    const int n = (int)n64;
    const int nrt = (m + kZM - 1) / kZM, nch = (m + kZC - 1) / kZC;
    char* p = (char*)scratch;
    __nv_bfloat16* Adig = (__nv_bfloat16*)p;
    p += (size_t)nrt * nch * kZDig * kZADig;
    __nv_bfloat16* Bdig = (__nv_bfloat16*)p;
    p += (size_t)nch * kZBChunk;
    int* ex = (int*)p;
    int* fy = ex + (size_t)nch * nrt * kZM;
    {
        a22_digits_kernel<<<dim3((unsigned)(nrt * kZM / 32), (unsigned)nch), 256, 0, st>>>(A, n, r1, m, nrt, nch, Adig, ex);
        note_launch();
        v_digits_kernel<<<(nch * (kZC / 8) * kZL + 127) / 128, 128, 0, st>>>(V, n, r1, m, nch, Bdig, fy);
        note_launch();
        BSE_CUDA(cudaGetLastError());
    }
    ZArgs z;
    z.Adig = Adig;
    z.Bdig = Bdig;
    z.ex = ex;
    z.fy = fy;
    z.zpart = zpart;
    z.m = m;
    z.nrt = nrt;
    z.nch = nch;
    z.nsplit = nsplit;
    z.status = status;
    z.spin = wait_limit(wait_polls, kMbarSpinLimit);
    BSE_CUDA(cudaFuncSetAttribute(zgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kZSmem));
    zgemm_tc_kernel<<<dim3(nrt, nsplit), kZWThreads, kZSmem, st>>>(z);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

}  // namespace bse
