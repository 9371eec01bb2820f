// Panel-end update of the blocked tridiagonal reduction on the tcgen05 tensor
// cores, accurate to about 2^-48 of its largest term (sm_103a).
//
// At the end of a panel of reflectors (V_l, W_l, l < 32) the trailing matrix
// (rows and columns >= k0, both triangles, double-float) receives
//
//   A -= sum_l (V_l W_l^H + W_l V_l^H) = X Y^H,   X = [V W], Y = [W V]   (n x 64 complex)
//
// a dense complex contraction with K = 64.  In real form, with K' = 128,
//   Re(X Y^H) = [Xr Xi] [Yr Yi]^T,   Im(X Y^H) = [Xr Xi] [-Yi Yr]^T,
// so X is stored once and each 32-column tile of Y in both forms, stacked as
// the 64 rows (N) of one MMA operand: one MMA gives the real and imaginary parts.
// Before the split, V_l is scaled by 2^g_l and W_l by 2^-g_l, with g_l half the
// difference of the exponents of their largest entries: the products V_l W_l^H
// and W_l V_l^H are unchanged (powers of two), and the 64 columns of a row come
// to comparable magnitudes.  (A reflector from a start vector of rounding-level
// size, e.g. the projection of a dark block, has |V_0| ~ 1e-17 and |W_0| ~ 1e17;
// unbalanced, such a column would set the scale of every row.)
// The double-float operands are then split exactly into digits: a row x of X (or
// Y) is scaled by 2^-e with 2^e above its largest element, rounded to 56 bits,
// q = rint(x 2^(56-e)), and written in balanced base 128,
//   q = sum_{k=0..7} d_k 2^(49-7k),   |d_0| <= 128, |d_k| <= 64,
// and the digits are stored pre-scaled, x_k = d_k 2^-7k, which bf16 holds exactly.
// A product x_k y_m is an integer below 2^14 times 2^-7(k+m), so for each
// g = k + m the sum over K' and over the pairs with that g is an integer below
// 2^24 times 2^-7g: exact in an FP32 accumulator of TMEM.  The groups g = 0..3
// accumulate exactly, one accumulator each; the pairs with 4 <= g <= 7 (weights
// below 2^-28 of the largest term) share a fifth accumulator, whose FP32
// rounding stays below 2^-48 of that term; pairs with g > 7 (below 2^-56) are
// left out.  Then
//   (X Y^H)_ri = 2^(e_r + f_i - 14) (G_0 + G_1 + G_2 + G_3 + G_rest),
// summed in double-float by the epilogue, scaled by the powers of two and
// subtracted from A in double-float.
//
// Layout: the digits of X (a 128-row tile) and of Y (a 32-row tile in both forms)
// are written by panel_digits_kernel in the tcgen05 core-matrix layout, tile
// after tile, so that one bulk copy brings a tile's operand.  A persistent kernel
// (one CTA of 4 warps per SM) takes a contiguous range of the 128 x 32 output
// tiles in column-tile-major order: the 8 digits of the Y tile (128 KB) stay in
// shared memory while its row tiles pass, the digits of X stream through a ring
// of three 32 KB slots, and one thread keeps the tensor pipe fed (the MMAs of
// digit k are queued before it waits for those of digit k - 1, whose slot then
// takes digit k + 2).  A tile's 5 x 64 accumulator columns are read back by all
// four warps (a warp per 32 TMEM lanes = rows) while the next digits land.
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

constexpr int kHM = 128;           // rows of an output tile (TMEM lanes, M of the MMA)
constexpr int kHN = 32;            // complex output columns of a tile
constexpr int kBN = 64;            // N of the MMA: the tile's rows of [Yr Yi], then of [-Yi Yr]
constexpr int kHK = 128;           // K of the real GEMM (64 complex terms: 32 reflectors, V and W)
constexpr int kDig = kDigits;      // digits per operand
constexpr int kExact = 4;          // digit-pair groups g < kExact accumulate exactly, one accumulator each
constexpr int kAcc = kExact + 1;   // accumulators per tile (the last one holds the groups g >= kExact)
constexpr int kSlots = 3;          // ring of X digit buffers
constexpr int kHThreads = 128;
constexpr uint32_t kHTmemCols = 512;                       // kAcc x kBN = 320 used
constexpr size_t kADigBytes = (size_t)kHM * kHK * 2;       // one digit of an X tile (32 KB)
constexpr size_t kBDigBytes = (size_t)kBN * kHK * 2;       // one digit of a Y tile, both forms (16 KB)
constexpr size_t kBTileBytes = kDig * kBDigBytes;          // the 8 digits of a Y tile (128 KB)
constexpr size_t kHerSmem = kBTileBytes + kSlots * kADigBytes + 1024;

// Exponents of the largest entries of V_l (block l) and W_l (block 32 + l) on rows
// [k0, n); kNoExp for a column of zeros
constexpr int kNoExp = -100000;
__global__ void panel_colexp_kernel(const cdf* __restrict__ V, const cdf* __restrict__ W, int n, int k0, int* cx) {
    __shared__ float s_m[kHThreads / 32];
    const int l = blockIdx.x & 31;
    const cdf* x = (blockIdx.x >= 32 ? W : V) + (size_t)l * n;
    float m = 0.f;
    for (int r = k0 + (int)threadIdx.x; r < n; r += blockDim.x) {
        const cdf z = __ldcg(x + r);
        m = fmaxf(m, fmaxf(fabsf(z.x), fabsf(z.z)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_m[w]);
        cx[blockIdx.x] = m > 0.f ? ilogbf(m) : kNoExp;
    }
}

// balance exponent g_l of reflector pair l: V_l is scaled by 2^g_l, W_l by 2^-g_l
__device__ __forceinline__ int balance_exp(const int* cx, int l) {
    const int ev = cx[l], ew = cx[32 + l];
    if (ev == kNoExp || ew == kNoExp) return 0;
    return max(-120, min(120, (ew - ev) >> 1));
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
    float v[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};   // Re, Im of column lane, then lane + 32
    if (live) {
        const cdf a = isx ? __ldcg(V + (size_t)lane * n + r) : __ldcg(W + (size_t)lane * n + r);
        const cdf b = isx ? __ldcg(W + (size_t)lane * n + r) : __ldcg(V + (size_t)lane * n + r);
        const int g = balance_exp(cx, lane);   // V_l scaled by 2^g, W_l by 2^-g (exact)
        const int ga = isx ? g : -g, gb = -ga;
        v[0][0] = scale_pow2(a.x, ga), v[0][1] = scale_pow2(a.y, ga);
        v[1][0] = scale_pow2(a.z, ga), v[1][1] = scale_pow2(a.w, ga);
        v[2][0] = scale_pow2(b.x, gb), v[2][1] = scale_pow2(b.y, gb);
        v[3][0] = scale_pow2(b.z, gb), v[3][1] = scale_pow2(b.w, gb);
    }
    float m = fmaxf(fmaxf(fabsf(v[0][0]), fabsf(v[1][0])), fmaxf(fabsf(v[2][0]), fabsf(v[3][0])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = exp_above_f(m);   // |x| < 2^e for every element of the row
    if (lane == 0) (isx ? ex : fy)[r] = e;
    float d[4][kDig];
#pragma unroll
    for (int j = 0; j < 4; ++j) df_digits8(v[j][0], v[j][1], e, d[j]);
    // K index: real parts of columns 0..63 at 0..63, imaginary parts at 64..127; digit k
    // stored as d_k 2^-7k (exact in bf16)
    const int kr0 = lane, kr1 = lane + 32, ki0 = 64 + lane, ki1 = 96 + lane;
    auto bf = [](float x) { return __float2bfloat16_rn(x); };
    if (isx) {
        const int rt = r / kHM, rr = r % kHM;
#pragma unroll
        for (int k = 0; k < kDig; ++k) {
            unsigned char* base = (unsigned char*)Adig + ((size_t)rt * kDig + k) * kADigBytes;   // [Xr Xi]
            *(__nv_bfloat16*)(base + tc::core_off(rr, kr0, kHK)) = bf(d[0][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, kr1, kHK)) = bf(d[2][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, ki0, kHK)) = bf(d[1][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, ki1, kHK)) = bf(d[3][k]);
        }
    } else {
        const int ct = r / kHN, rr = r % kHN;
#pragma unroll
        for (int k = 0; k < kDig; ++k) {
            unsigned char* base = (unsigned char*)Bdig + ((size_t)ct * kDig + k) * kBDigBytes;
            // row rr: [Yr Yi]; row rr + 32: [-Yi Yr]
            *(__nv_bfloat16*)(base + tc::core_off(rr, kr0, kHK)) = bf(d[0][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, kr1, kHK)) = bf(d[2][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, ki0, kHK)) = bf(d[1][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr, ki1, kHK)) = bf(d[3][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr + kHN, kr0, kHK)) = bf(-d[1][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr + kHN, kr1, kHK)) = bf(-d[3][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr + kHN, ki0, kHK)) = bf(d[0][k]);
            *(__nv_bfloat16*)(base + tc::core_off(rr + kHN, ki1, kHK)) = bf(d[2][k]);
        }
    }
}

struct HerArgs {
    cdf* A;                            // n x n column-major, double-float
    const __nv_bfloat16* Adig;         // [nrt][8][128 x 128] core-matrix layout
    const __nv_bfloat16* Bdig;         // [nct][8][64 x 128]
    const int* ex;                     // [nrt*128] row exponents of X
    const int* fy;                     // [nct*32] row exponents of Y
    int n, k0, rt0, ct0, ntr, ntc;     // trailing block from k0; tiles rt0.., ct0.. (ntr x ntc of them)
    int resident_from;                 // columns below it are streamed (evict-first loads and stores)
    int* status;                       // raised when a bounded wait gives up
    long spin;                         // polls of an mbarrier wait before it gives up
};

// DF sum of the five accumulators of one output (exact FP32 values)
__device__ __forceinline__ float2 her_sum(const uint32_t (&v)[kAcc][8], int j) {
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

// Persistent: CTA b takes the tiles [T b / G, T (b + 1) / G) of the column-tile-major order
// (t = ctl * ntr + rtl), with warp-specialised roles: warp 4 (one lane) copies a tile's Y
// digits when its column tile changes (once the MMAs of the previous tile are done) and streams
// the 8 X digits of each tile through three slots as they free up; warp 5 (one lane) issues the
// MMAs as operands land, once the epilogue of the previous tile has released TMEM; warps 0-3
// (a warp per 32 TMEM lanes = rows) read the accumulators back and update A.  X item j = digit
// j % 8 of tile j / 8 uses slot j % 3 (its copy the (j / 3)-th completion of mb_full[slot], its
// MMAs the (j / 3)-th commit to mb_empty[slot]); mb_acc and mb_free complete once per tile,
// mb_y once per Y copy.  TMEM column of accumulator c, output column i of the tile: c * 64 + i
// (real part), c * 64 + 32 + i (imaginary part).
constexpr int kHWThreads = 192;
__global__ void __launch_bounds__(kHWThreads, 1) panel_update_tc_kernel(HerArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* Bs = smem;                                  // 8 digits of the Y tile (both forms)
    unsigned char* As = smem + kBTileBytes;                    // kSlots digit buffers of X tiles
    __shared__ __align__(8) uint64_t mb_y, mb_full[kSlots], mb_empty[kSlots], mb_acc, mb_free, mb_fin;
    __shared__ uint32_t slot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&mb_y, 1);
        tc::mbar_init(&mb_acc, 1);
        tc::mbar_init(&mb_free, 4);
        tc::mbar_init(&mb_fin, 1);
        for (int i = 0; i < kSlots; ++i) {
            tc::mbar_init(&mb_full[i], 1);
            tc::mbar_init(&mb_empty[i], 1);
        }
        s_abort = 0;
    }
    if (warp == 0) tc::tmem_alloc(&slot, kHTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = slot;
    volatile int* abort = &s_abort;
    const int64_t T = (int64_t)a.ntr * a.ntc;
    const int t_begin = (int)(T * blockIdx.x / gridDim.x), t_end = (int)(T * (blockIdx.x + 1) / gridDim.x);
    const int ntl = t_end - t_begin;
    auto tile_ct = [&](int tl) { return a.ct0 + (t_begin + tl) / a.ntr; };
    auto tile_rt = [&](int tl) { return a.rt0 + (t_begin + tl) % a.ntr; };
    auto fail_now = [&]() {
        *abort = 1;
        atomicExch(a.status, 1);
    };
    if (warp == 4) {
        if (lane == 0) {   // producer
            int last[kSlots] = {-1, -1, -1}, ys = 0, cur_ct = -1;
            bool ok = true;
            for (int tl = 0; tl < ntl && ok; ++tl) {
                const int ct = tile_ct(tl), rt = tile_rt(tl);
                if (ct != cur_ct) {   // the MMAs of the previous tile are done: the Y buffer is free
                    if (tl > 0 && !(ok = ws_wait(&mb_acc, (uint32_t)((tl - 1) & 1), a.spin, abort))) break;
                    tc::mbar_expect_tx(&mb_y, (uint32_t)kBTileBytes);
                    tc::bulk_g2s(Bs, (const unsigned char*)a.Bdig + (size_t)ct * kBTileBytes, (uint32_t)kBTileBytes,
                                 &mb_y);
                    ++ys;
                    cur_ct = ct;
                }
                for (int k = 0; k < kDig; ++k) {
                    const int j = tl * kDig + k, sl = j % kSlots;
                    if (j >= kSlots &&
                        !(ok = ws_wait(&mb_empty[sl], (uint32_t)(((j - kSlots) / kSlots) & 1), a.spin, abort)))
                        break;
                    tc::mbar_expect_tx(&mb_full[sl], (uint32_t)kADigBytes);
                    tc::bulk_g2s(As + sl * kADigBytes,
                                 (const unsigned char*)a.Adig + ((size_t)rt * kDig + k) * kADigBytes,
                                 (uint32_t)kADigBytes, &mb_full[sl]);
                    last[sl] = j;
                }
            }
            if (!ok) fail_now();
            for (int sl = 0; sl < kSlots; ++sl)
                if (last[sl] >= 0) tc::mbar_wait(&mb_full[sl], (uint32_t)((last[sl] / kSlots) & 1), kMbarSpinLimit);
            if (ys > 0) tc::mbar_wait(&mb_y, (uint32_t)((ys - 1) & 1), kMbarSpinLimit);
        }
    } else if (warp == 5) {
        if (lane == 0) {   // MMA issuer
            const uint32_t idesc = tc::idesc_f16(kHM, kBN, 1);
            const uint32_t lbo = 128, sbo = (uint32_t)(kHK / 8) * 128;
            int yw = 0, cur_ct = -1;
            bool ok = true;
            for (int tl = 0; tl < ntl && ok; ++tl) {
                const int ct = tile_ct(tl);
                if (ct != cur_ct) {
                    if (!(ok = ws_wait(&mb_y, (uint32_t)(yw & 1), a.spin, abort))) break;
                    ++yw;
                    cur_ct = ct;
                }
                if (tl > 0 && !(ok = ws_wait(&mb_free, (uint32_t)((tl - 1) & 1), a.spin, abort))) break;
                tc::fence_after();
                for (int k = 0; k < kDig; ++k) {
                    const int j = tl * kDig + k, sl = j % kSlots;
                    if (!(ok = ws_wait(&mb_full[sl], (uint32_t)((j / kSlots) & 1), a.spin, abort))) break;
                    tc::fence_after();
                    const uint64_t ad = tc::smem_desc(tc::smem_u32(As + sl * kADigBytes), lbo, sbo);
                    for (int m = 0; m + k < kDig; ++m) {
                        const int g = k + m, acc = g < kExact ? g : kExact;
                        const bool first = k == 0 && (g < kExact || m == kExact);
                        const uint64_t bd = tc::smem_desc(tc::smem_u32(Bs + m * kBDigBytes), lbo, sbo);
                        const uint32_t d = tmem + (uint32_t)(acc * kBN);
#pragma unroll
                        for (int ks = 0; ks < kHK / 16; ++ks)   // 16 K per MMA: 256 bytes, 16 descriptor units
                            tc::mma_f16(d, ad + (uint64_t)(ks * 16), bd + (uint64_t)(ks * 16), idesc,
                                        (first && ks == 0) ? 0u : 1u);
                    }
                    tc::mma_commit(&mb_empty[sl]);
                }
                if (ok) tc::mma_commit(&mb_acc);
            }
            if (!ok) fail_now();
            tc::mma_commit(&mb_fin);   // every MMA issued has completed before TMEM is released
            tc::mbar_wait(&mb_fin, 0u, kMbarSpinLimit);
        }
    } else {   // epilogue warps 0-3
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
        for (int tl = 0; tl < ntl; ++tl) {
            const int ct = tile_ct(tl), rt = tile_rt(tl);
            const int r = rt * kHM + warp * 32 + lane;
            const bool rlive = r >= a.k0 && r < a.n;
            auto load_chunk = [&](int c0, cdf* q) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int i = ct * kHN + c0 + j;
                    const cdf* src = a.A + (size_t)i * a.n + r;
                    q[j] = rlive && i >= a.k0 && i < a.n ? (i < a.resident_from ? __ldcs(src) : __ldcg(src))
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            };
            cdf qa[8], qb[8];
            load_chunk(0, qa);   // loads while the MMAs run
            if (!ws_wait(&mb_acc, (uint32_t)(tl & 1), a.spin, abort)) {
                fail_now();
                break;
            }
            tc::fence_after();
            const int er = rlive ? __ldg(a.ex + r) : 0;
            auto finish_chunk = [&](int c0, const cdf* q) {
                uint32_t vr[kAcc][8], vi[kAcc][8];
#pragma unroll
                for (int c = 0; c < kAcc; ++c) {
                    tc::tmem_ld8_async(tmem + lane_off + (uint32_t)(c * kBN + c0), vr[c]);
                    tc::tmem_ld8_async(tmem + lane_off + (uint32_t)(c * kBN + kHN + c0), vi[c]);
                }
#pragma unroll
                for (int c = 0; c < kAcc; ++c) {
                    tc::tmem_ld_wait(vr[c]);
                    tc::tmem_ld_wait(vi[c]);
                }
                if (rlive)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int i = ct * kHN + c0 + j;
                        if (i < a.k0 || i >= a.n) continue;
                        const float sc = ldexpf(1.f, er + __ldg(a.fy + i) - 14);
                        const float2 sr = her_sum(vr, j), si = her_sum(vi, j);
                        const float2 re = df_add(make_float2(q[j].x, q[j].y), make_float2(-sr.x * sc, -sr.y * sc));
                        const float2 im = df_add(make_float2(q[j].z, q[j].w), make_float2(-si.x * sc, -si.y * sc));
                        const cdf out = make_float4(re.x, re.y, im.x, im.y);
                        if (i < a.resident_from)
                            __stcs(a.A + (size_t)i * a.n + r, out);
                        else
                            a.A[(size_t)i * a.n + r] = out;
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
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&mb_free)) : "memory");
        }
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

int launch_panel_update_tc(cdf* A, int64_t n, int k0, int resident_from, const cdf* V, const cdf* W, void* scratch,
                           int* status, cudaStream_t st, long wait_polls) {
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
    h.resident_from = resident_from;
    h.status = status;
    h.spin = wait_limit(wait_polls, kMbarSpinLimit);
    BSE_CUDA(cudaFuncSetAttribute(panel_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHerSmem));
    int dev = 0, sms = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ntiles = (int64_t)h.ntr * h.ntc;
    const int grid = (int)std::min<int64_t>(sms, ntiles);
    panel_update_tc_kernel<<<grid, kHWThreads, kHerSmem, st>>>(h);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

}  // namespace bse
