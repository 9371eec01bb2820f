// Panel-end update of the blocked tridiagonal reduction on the tcgen05 tensor
// cores, exact to about 2^-50 of its terms (sm_103a).
//
// At the end of a panel of reflectors (V_l, W_l, l < 32) the trailing matrix
// (rows and columns >= k0, both triangles, double-float) receives
//
//   A -= sum_l (V_l W_l^H + W_l V_l^H) = X Y^H,   X = [V W], Y = [W V]   (n x 64 complex)
//
// a dense complex contraction with K = 64.  In real form, with K' = 128,
//   Re(X Y^H) = [Xr Xi] [Yr Yi]^T,   Im(X Y^H) = [Xi -Xr] [Yr Yi]^T.
// Before the split, V_l is scaled by 2^g_l and W_l by 2^-g_l, with g_l half the
// difference of the exponents of their largest entries: the products V_l W_l^H
// and W_l V_l^H are unchanged (powers of two), and the 64 columns of a row come
// to comparable magnitudes.  (A reflector from a start vector of rounding-level
// size, e.g. the projection of a dark block, has |V_0| ~ 1e-17 and |W_0| ~ 1e17;
// unbalanced, such a column would set the scale of every row.)
// The double-float operands are then split exactly into integer digits: a row x
// of X (or Y) is scaled by 2^-e with 2^e above its largest element, rounded to 56
// bits, q = rint(x 2^(56-e)), and written in balanced base 128,
//   q = sum_{k=0..7} d_k 2^(49-7k),   |d_0| <= 128, |d_k| <= 64,
// each digit an integer that bf16 holds exactly.  A product of two digits is
// an integer below 2^14, a sum of 128 of them below 2^21, and the sum of the
// up to 8 digit pairs (k, m) with the same k + m below 2^24: every partial GEMM
// is exact in the FP32 accumulators of TMEM.  Pairs with k + m <= 7 are kept
// (the others weigh below 2^-112 of the largest term), so that
//   (X Y^H)_ri = 2^(e_r + f_i) sum_{g=0..7} 2^(-7g - 14) G_g[r,i],
//   G_g = sum_{k+m=g} D^X_k (D^Y_m)^T,
// and the result carries the 56-bit rounding of the operands only, below the
// reduction's double-float roundoff.  The epilogue sums the eight exact FP32
// groups in double-float, scales by the two powers of two and subtracts the
// result from A in double-float.
//
// Layout: the digits of X (both real operands of a 128-row tile) and of Y (a
// 32-row tile) are written by panel_digits_kernel in the tcgen05 core-matrix
// layout, tile after tile, so that one bulk copy brings a tile's operand.  A
// persistent kernel (one CTA of 4 warps per SM) takes 128 x 32 output tiles of
// the trailing block; per tile its 512 TMEM columns hold the 8 groups x
// (real, imaginary) x 32 columns, the 8 digits of Y stay in shared memory
// (64 KB), the digits of X stream through two 64 KB buffers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "dfloat.h"
#include "grid_sync.h"
#include "internal.h"
#include "tc_ptx.h"

namespace bse {

namespace {

constexpr int kHM = 128;           // rows of an output tile (TMEM lanes, M of the MMA)
constexpr int kHN = 32;            // columns of an output tile (N of the MMA)
constexpr int kHK = 128;           // K of the real GEMM (64 complex terms: 32 reflectors, V and W)
constexpr int kDig = 8;            // digits per operand
constexpr int kHThreads = 128;
constexpr uint32_t kHTmemCols = 512;
constexpr size_t kADigBytes = (size_t)2 * kHM * kHK * 2;   // one digit of an X tile: real and imaginary operands
constexpr size_t kBDigBytes = (size_t)kHN * kHK * 2;       // one digit of a Y tile
constexpr size_t kBTileBytes = kDig * kBDigBytes;          // the 8 digits of a Y tile (64 KB)
constexpr size_t kHerSmem = kBTileBytes + 2 * kADigBytes + 1024;

__device__ __forceinline__ double cdf_re(cdf z) { return (double)z.x + (double)z.y; }
__device__ __forceinline__ double cdf_im(cdf z) { return (double)z.z + (double)z.w; }

// balanced base-128 digits of q (|q| <= 2^56): d_0 .. d_7, weights 2^49 .. 2^0
__device__ __forceinline__ void digits8(long long q, float* d) {
#pragma unroll
    for (int k = 0; k < kDig; ++k) {
        const int sh = 49 - 7 * k;
        long long dk;
        if (sh > 0) {
            dk = (q + (1ll << (sh - 1))) >> sh;   // nearest integer (arithmetic shift floors)
            q -= dk << sh;
        } else {
            dk = q;
        }
        d[k] = (float)dk;
    }
}

// 2^p as a double (p within the normal range)
__device__ __forceinline__ double pow2d(int p) { return __longlong_as_double((long long)(1023 + p) << 52); }

// Exponents of the largest entries of V_l (block l) and W_l (block 32 + l) on rows
// [k0, n); kNoExp for a column of zeros
constexpr int kNoExp = -100000;
__global__ void panel_colexp_kernel(const cdf* __restrict__ V, const cdf* __restrict__ W, int n, int k0, int* cx) {
    __shared__ double s_m[kHThreads / 32];
    const int l = blockIdx.x & 31;
    const cdf* x = (blockIdx.x >= 32 ? W : V) + (size_t)l * n;
    double m = 0.0;
    for (int r = k0 + (int)threadIdx.x; r < n; r += blockDim.x) {
        const cdf z = __ldcg(x + r);
        m = fmax(m, fmax(fabs(cdf_re(z)), fabs(cdf_im(z))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_m[w]);
        cx[blockIdx.x] = m > 0.0 ? ilogb(m) : kNoExp;
    }
}

// balance exponent g_l of reflector pair l: V_l is scaled by 2^g_l, W_l by 2^-g_l
__device__ __forceinline__ int balance_exp(const int* cx, int l) {
    const int ev = cx[l], ew = cx[32 + l];
    if (ev == kNoExp || ew == kNoExp) return 0;
    return max(-500, min(500, (ew - ev) >> 1));
}

// One warp per row of X (rows rt0*128 <= r < nrt*128) or of Y (rows ct0*32 <= i < nct*32,
// after the X rows): the rows of the tiles the update reads.  Rows outside [k0, n) get zero digits.  X row r: X[r,c] = V_c[r] (c < 32), W_{c-32}[r];
// Y row i: Y[i,c] = W_c[i] (c < 32), V_{c-32}[i].  Lane c holds columns c and c + 32.
__global__ void panel_digits_kernel(const cdf* __restrict__ V, const cdf* __restrict__ W, int n, int k0, int rt0,
                                    int nrt, int ct0, int nct, const int* __restrict__ cx, __nv_bfloat16* Adig,
                                    __nv_bfloat16* Bdig, int* ex, int* fy) {
    const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int nx = (nrt - rt0) * kHM, ny = (nct - ct0) * kHN;
    if (gw >= nx + ny) return;
    const bool isx = gw < nx;
    const int r = isx ? rt0 * kHM + gw : ct0 * kHN + (gw - nx);
    const bool live = r >= k0 && r < n;
    double v[4] = {0.0, 0.0, 0.0, 0.0};   // Re, Im of column lane, then of column lane + 32
    if (live) {
        const cdf a = isx ? __ldcg(V + (size_t)lane * n + r) : __ldcg(W + (size_t)lane * n + r);
        const cdf b = isx ? __ldcg(W + (size_t)lane * n + r) : __ldcg(V + (size_t)lane * n + r);
        const int g = balance_exp(cx, lane);
        const double sv = pow2d(g), sw = pow2d(-g);   // V_l and W_l balanced (exact)
        const double sa = isx ? sv : sw, sb = isx ? sw : sv;
        v[0] = cdf_re(a) * sa;
        v[1] = cdf_im(a) * sa;
        v[2] = cdf_re(b) * sb;
        v[3] = cdf_im(b) * sb;
    }
    double m = fmax(fmax(fabs(v[0]), fabs(v[1])), fmax(fabs(v[2]), fabs(v[3])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = m > 0.0 ? ilogb(m) + 1 : 0;   // |x| < 2^e for every element of the row
    if (lane == 0) (isx ? ex : fy)[r] = e;
    const double sc = pow2d(56 - e);
    float d[4][kDig];
#pragma unroll
    for (int j = 0; j < 4; ++j) digits8(__double2ll_rn(v[j] * sc), d[j]);
    // K index: real parts of columns 0..63 at 0..63, imaginary parts at 64..127
    const int kr0 = lane, kr1 = lane + 32, ki0 = 64 + lane, ki1 = 96 + lane;
    if (isx) {
        const int rt = r / kHM, rr = r % kHM;
#pragma unroll
        for (int k = 0; k < kDig; ++k) {
            unsigned char* base = (unsigned char*)Adig + ((size_t)rt * kDig + k) * kADigBytes;
            unsigned char* re = base;                                 // [Xr Xi]
            unsigned char* im = base + (size_t)kHM * kHK * 2;         // [Xi -Xr]
            *(__nv_bfloat16*)(re + tc::core_off(rr, kr0, kHK)) = __float2bfloat16_rn(d[0][k]);
            *(__nv_bfloat16*)(re + tc::core_off(rr, kr1, kHK)) = __float2bfloat16_rn(d[2][k]);
            *(__nv_bfloat16*)(re + tc::core_off(rr, ki0, kHK)) = __float2bfloat16_rn(d[1][k]);
            *(__nv_bfloat16*)(re + tc::core_off(rr, ki1, kHK)) = __float2bfloat16_rn(d[3][k]);
            *(__nv_bfloat16*)(im + tc::core_off(rr, kr0, kHK)) = __float2bfloat16_rn(d[1][k]);
            *(__nv_bfloat16*)(im + tc::core_off(rr, kr1, kHK)) = __float2bfloat16_rn(d[3][k]);
            *(__nv_bfloat16*)(im + tc::core_off(rr, ki0, kHK)) = __float2bfloat16_rn(-d[0][k]);
            *(__nv_bfloat16*)(im + tc::core_off(rr, ki1, kHK)) = __float2bfloat16_rn(-d[2][k]);
        }
    } else {
        const int ct = r / kHN, rr = r % kHN;
#pragma unroll
        for (int k = 0; k < kDig; ++k) {
            unsigned char* base = (unsigned char*)Bdig + ((size_t)ct * kDig + k) * kBDigBytes;   // [Yr Yi]
            *(__nv_bfloat16*)(base + tc::core_off(rr, kr0, kHK)) = __float2bfloat16_rn(d[0][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, kr1, kHK)) = __float2bfloat16_rn(d[2][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, ki0, kHK)) = __float2bfloat16_rn(d[1][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, ki1, kHK)) = __float2bfloat16_rn(d[3][k]);
        }
    }
}

struct HerArgs {
    cdf* A;                            // n x n column-major, double-float
    const __nv_bfloat16* Adig;         // [nrt][8][2][128 x 128] core-matrix layout
    const __nv_bfloat16* Bdig;         // [nct][8][32 x 128]
    const int* ex;                     // [nrt*128] row exponents of X
    const int* fy;                     // [nct*32] row exponents of Y
    int n, k0, rt0, ct0, ntr, ntc;     // trailing block from k0; tiles rt0.., ct0.. (ntr x ntc of them)
    int* status;                       // raised when a bounded wait gives up
    long spin;                         // polls of an mbarrier wait before it gives up
};

// Persistent: output tiles (rt, ct) in row-tile-major order, blockIdx.x + j gridDim.x.
// TMEM column of group g, part p (0 real, 1 imaginary), output column c: (p * 8 + g) * 32 + c.
__global__ void __launch_bounds__(kHThreads, 1) panel_update_tc_kernel(HerArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* Bs = smem;                                  // 8 digits of the Y tile
    unsigned char* As = smem + kBTileBytes;                    // two digit buffers of the X tile
    __shared__ __align__(8) uint64_t mb_b, mb_a[2], mb_m[2];
    __shared__ uint32_t slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&mb_b, 1);
        tc::mbar_init(&mb_a[0], 1);
        tc::mbar_init(&mb_a[1], 1);
        tc::mbar_init(&mb_m[0], 1);
        tc::mbar_init(&mb_m[1], 1);
    }
    if (warp == 0) tc::tmem_alloc(&slot, kHTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = slot;
    // phases issued (copies started, MMAs committed) and waited for, per mbarrier
    uint32_t ib = 0, pb = 0, ia[2] = {0, 0}, pa[2] = {0, 0}, im[2] = {0, 0}, pm[2] = {0, 0};
    const uint32_t idesc = tc::idesc_f16(kHM, kHN, 1);
    const uint32_t lbo = 128, sbo = (uint32_t)(kHK / 8) * 128;
    bool ok = true;
    // a bounded wait; on giving up the awaited operation is still let finish (default limit)
    auto wait = [&](uint64_t* mb, uint32_t& ph) {
        const bool got = tc::mbar_wait(mb, ph & 1u, a.spin);
        if (!got) tc::mbar_wait(mb, ph & 1u, kMbarSpinLimit);
        ++ph;
        return got;
    };
    const int ntiles = a.ntr * a.ntc;
    // bulk copies of a tile's Y digits and of its first two X digits (tid 0 issues, all count)
    auto issue_tile = [&](int t) {
        const int rt = a.rt0 + t / a.ntc, ct = a.ct0 + t % a.ntc;
        const unsigned char* ag = (const unsigned char*)a.Adig + (size_t)rt * kDig * kADigBytes;
        if (tid == 0) {
            tc::mbar_expect_tx(&mb_b, (uint32_t)kBTileBytes);
            tc::bulk_g2s(Bs, (const unsigned char*)a.Bdig + (size_t)ct * kBTileBytes, (uint32_t)kBTileBytes, &mb_b);
            for (int b = 0; b < 2; ++b) {
                tc::mbar_expect_tx(&mb_a[b], (uint32_t)kADigBytes);
                tc::bulk_g2s(As + b * kADigBytes, ag + b * kADigBytes, (uint32_t)kADigBytes, &mb_a[b]);
            }
        }
        ++ib;
        ++ia[0];
        ++ia[1];
    };
    if ((int)blockIdx.x < ntiles) issue_tile(blockIdx.x);
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int rt = a.rt0 + t / a.ntc, ct = a.ct0 + t % a.ntc;
        const unsigned char* ag = (const unsigned char*)a.Adig + (size_t)rt * kDig * kADigBytes;
        // this thread's row of the output tile; its first 8 entries of A load while the MMAs run
        const int r = rt * kHM + warp * 32 + lane;
        const bool rlive = r >= a.k0 && r < a.n;
        auto load_chunk = [&](int c0, cdf* q) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int i = ct * kHN + c0 + j;
                q[j] = rlive && i >= a.k0 && i < a.n ? __ldcg(a.A + (size_t)i * a.n + r) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        cdf qa[8], qb[8];
        load_chunk(0, qa);
        ok = __syncthreads_and(wait(&mb_b, pb)) != 0;
        for (int k = 0; k < kDig && ok; ++k) {
            const int b = k & 1;
            ok = __syncthreads_and(wait(&mb_a[b], pa[b])) != 0;
            if (!ok) break;
            tc::fence_after();
            if (tid == 0) {
                const uint32_t a0 = tc::smem_u32(As + b * kADigBytes), b0 = tc::smem_u32(Bs);
                for (int m = 0; m + k < kDig; ++m) {
                    const int g = k + m;
                    for (int part = 0; part < 2; ++part) {
                        const uint32_t d = tmem + (uint32_t)((part * kDig + g) * kHN);
                        const uint32_t ab = a0 + (uint32_t)(part * kHM * kHK * 2);
                        const uint32_t bb = b0 + (uint32_t)(m * kBDigBytes);
                        for (int ks = 0; ks < kHK / 16; ++ks)
                            tc::mma_f16(d, tc::smem_desc(ab + ks * 256, lbo, sbo), tc::smem_desc(bb + ks * 256, lbo, sbo),
                                        idesc, (k | ks) != 0);
                    }
                }
                tc::mma_commit(&mb_m[b]);
            }
            ++im[b];
            if (k + 2 < kDig) {   // the buffer takes digit k + 2 once digit k's MMAs are done
                ok = __syncthreads_and(wait(&mb_m[b], pm[b])) != 0;
                if (ok) {
                    if (tid == 0) {
                        tc::mbar_expect_tx(&mb_a[b], (uint32_t)kADigBytes);
                        tc::bulk_g2s(As + b * kADigBytes, ag + (size_t)(k + 2) * kADigBytes, (uint32_t)kADigBytes,
                                     &mb_a[b]);
                    }
                    ++ia[b];
                }
            }
        }
        if (!ok) break;
        // the MMAs of digits 6 and 7
        {
            const bool w0 = wait(&mb_m[0], pm[0]);
            const bool w1 = wait(&mb_m[1], pm[1]);
            ok = __syncthreads_and(w0 && w1) != 0;
        }
        if (!ok) break;
        tc::fence_after();
        // shared memory is free: the next tile's copies land during the epilogue
        if (t + (int)gridDim.x < ntiles) issue_tile(t + gridDim.x);
        // epilogue, 8 columns at a time (the next 8 entries of A loading meanwhile): the eight
        // exact groups read together, summed in double-float, scaled by 2^(e_r + f_i), subtracted
        const int er = rlive ? __ldg(a.ex + r) : 0;
        auto finish_chunk = [&](int c0, const cdf* q) {
            float2 acc[2][8];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                uint32_t v[kDig][8];
#pragma unroll
                for (int g = 0; g < kDig; ++g)
                    tc::tmem_ld8_async(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((p * kDig + g) * kHN + c0), v[g]);
#pragma unroll
                for (int g = 0; g < kDig; ++g) tc::tmem_ld_wait(v[g]);
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[p][j] = make_float2(0.f, 0.f);
#pragma unroll
                for (int g = 0; g < kDig; ++g) {
                    const float w = __int_as_float((127 - 7 * g - 14) << 23);   // 2^(-7g - 14), exact
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[p][j] = df_add(acc[p][j], make_float2(__uint_as_float(v[g][j]) * w, 0.f));
                }
            }
            if (rlive)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int i = ct * kHN + c0 + j;
                    if (i < a.k0 || i >= a.n) continue;
                    const float sc = ldexpf(1.f, er + __ldg(a.fy + i));
                    const float2 re = df_add(make_float2(q[j].x, q[j].y), make_float2(-acc[0][j].x * sc, -acc[0][j].y * sc));
                    const float2 im = df_add(make_float2(q[j].z, q[j].w), make_float2(-acc[1][j].x * sc, -acc[1][j].y * sc));
                    a.A[(size_t)i * a.n + r] = make_float4(re.x, re.y, im.x, im.y);
                }
        };
        load_chunk(8, qb);
        finish_chunk(0, qa);
        load_chunk(16, qa);
        finish_chunk(8, qb);
        load_chunk(24, qb);
        finish_chunk(16, qa);
        finish_chunk(24, qb);
        tc::fence_before();
        __syncthreads();   // TMEM is reused by the next tile
        tc::fence_after();
    }
    if (!ok) {
        // a wait gave up: let every copy and MMA still in flight finish (the default limit)
        // before the CTA frees its tensor memory and exits
        while (pb < ib) {
            tc::mbar_wait(&mb_b, pb & 1u, kMbarSpinLimit);
            ++pb;
        }
        for (int b = 0; b < 2; ++b) {
            while (pa[b] < ia[b]) {
                tc::mbar_wait(&mb_a[b], pa[b] & 1u, kMbarSpinLimit);
                ++pa[b];
            }
            while (pm[b] < im[b]) {
                tc::mbar_wait(&mb_m[b], pm[b] & 1u, kMbarSpinLimit);
                ++pm[b];
            }
        }
        if (tid == 0) atomicExch(a.status, 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kHTmemCols);
}

}  // namespace

size_t panel_update_tc_bytes(int64_t n) {
    const int64_t nrt = (n + kHM - 1) / kHM, nct = (n + kHN - 1) / kHN;
    return (size_t)nrt * kDig * kADigBytes + (size_t)nct * kBTileBytes + sizeof(int) * (size_t)(nrt * kHM + nct * kHN) +
           sizeof(int) * 64 + 4096;
}

int launch_panel_update_tc(cdf* A, int64_t n, int k0, const cdf* V, const cdf* W, void* scratch, int* status,
                           cudaStream_t st, long wait_polls) {
    if (k0 >= n) return BSE_OK;
    const int nrt = (int)((n + kHM - 1) / kHM), nct = (int)((n + kHN - 1) / kHN);
    const int rt0 = k0 / kHM, ct0 = k0 / kHN;
    char* p = (char*)scratch;
    __nv_bfloat16* Adig = (__nv_bfloat16*)p;
    p += (size_t)nrt * kDig * kADigBytes;
    __nv_bfloat16* Bdig = (__nv_bfloat16*)p;
    p += (size_t)nct * kBTileBytes;
    int* ex = (int*)p;
    int* fy = ex + (size_t)nrt * kHM;
    int* cx = fy + (size_t)nct * kHN;
    // balance exponents of the reflector pairs, then the digits of the rows the tiles read
    // (from the first tile row / column on)
    panel_colexp_kernel<<<64, kHThreads, 0, st>>>(V, W, (int)n, k0, cx);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    {
        const int64_t warps = (int64_t)(nrt - rt0) * kHM + (int64_t)(nct - ct0) * kHN;
        panel_digits_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(V, W, (int)n, k0, rt0, nrt, ct0, nct,
                                                                                cx, Adig, Bdig, ex, fy);
        note_launch();
        BSE_CUDA(cudaGetLastError());
    }
    HerArgs h;
    h.A = A;
    h.Adig = Adig;
    h.Bdig = Bdig;
    h.ex = ex;
    h.fy = fy;
    h.n = (int)n;
    h.k0 = k0;
    h.rt0 = rt0;
    h.ct0 = ct0;
    h.ntr = nrt - rt0;
    h.ntc = nct - ct0;
    h.status = status;
    h.spin = wait_limit(wait_polls, kMbarSpinLimit);
    BSE_CUDA(cudaFuncSetAttribute(panel_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHerSmem));
    int dev = 0, sms = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ntiles = (int64_t)h.ntr * h.ntc;
    const int grid = (int)std::min<int64_t>(sms, ntiles);
    panel_update_tc_kernel<<<grid, kHThreads, kHerSmem, st>>>(h);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

}  // namespace bse
