// Rotated direct-term blocks (Eq. Wtrafo): the direct term of a k pair
// (k, k') follows from the one of the symmetry-equivalent seed pair
// (s k, s k') by band rotations, since Gamma~(s) commutes with K^d:
//
//   K^d(k, k') = G(s,k)^dagger K^d(sk, sk') G(s,k'),
//   G(s,k)[(v1,c1),(v,c)] = Gamma(s)_{kc}^{sk c1} conj(Gamma(s)_{kv}^{sk v1})   (Eq. Ttilde)
//
// with Gamma(s) block-diagonal over the degenerate multiplets (Eq. Ts), so
// each element is a sum over at most 3 x 3 terms on either side.  The seed
// block is already in the tile arena; each element of the rotated block is
// written to its place in the tile (with its conjugate transpose when the
// tile is a diagonal star pair).  The kernel moves data: one read of the
// seed element per term and one or two writes.
#include <cuda_runtime.h>

#include "internal.h"

namespace bse {

namespace {

template <typename R>
struct C2r;
template <>
struct C2r<double> {
    using T = double2;
};
template <>
struct C2r<float> {
    using T = float2;
};

template <typename V>
__device__ __forceinline__ V cm(V a, V b) {   // a b
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename V>
__device__ __forceinline__ V cmc(V a, V b) {  // a conj(b)
    V r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}

// One warp per rotated pair, kRotWarps pairs per CTA (warp-level synchronisation
// only, so a pair's latency chain overlaps the other pairs').  Phase 1: for every
// row (v c) at k the factors L = Gamma_v(k)[v1][v] conj(Gamma_c(k)[c1][c]) with the
// seed rows (v1 c1) of its multiplets, and for every column (v' c') at k' the
// factors R = Gamma_c(k')[c2][c'] conj(Gamma_v(k')[v2][v']) with the seed columns,
// into the warp's part of shared memory (at most 9 terms each; one at a general k).
// Phase 2: out[(v c), (v' c')] = sum L S[(v1 c1), (v2 c2)] R, the seed element read
// from the tile arena, written to the block and to its mirror; where every
// multiplet of both sides is a single band (most k) the one-term form runs with
// several elements' loads in flight per lane.
constexpr int kMaxTerms = 9;
constexpr int kRotWarps = 8;

// shared memory of one warp: factors [2][B][kMaxTerms], seed indices [2][B][kMaxTerms], counts [2][B]
__host__ __device__ constexpr size_t rot_warp_bytes(int B, size_t vsize) {
    return (size_t)2 * B * kMaxTerms * (vsize + sizeof(int)) + sizeof(int) * 2 * (size_t)B;
}

template <typename R, bool kBatch>
__global__ void __launch_bounds__(kRotWarps * 32) rotate_kernel(const RotSys* __restrict__ systems,
                                                                const __grid_constant__ RotSys one,
                                                                const RotTask* __restrict__ tasks, int64_t ntasks,
                                                                int bstride, typename C2r<R>::T* X) {
    using V = typename C2r<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ti = (int64_t)blockIdx.x * kRotWarps + wid;
    if (ti >= ntasks) return;   // warp-uniform: no CTA-wide barrier follows
    const RotTask t = tasks[ti];
    const RotSys& Y = kBatch ? systems[t.flags >> 1] : one;
    const int nv = Y.nv, nc = Y.nc, nb = Y.nb, B = nv * nc;
    // the warps' parts are laid out for the launch's largest block (bstride >= B): the
    // instances of a batch may differ in B
    unsigned char* wbase = smem_raw + (size_t)wid * rot_warp_bytes(bstride, sizeof(V));
    V* fac = (V*)wbase;                                  // [2][B][kMaxTerms]
    int* idx = (int*)(fac + 2 * B * kMaxTerms);          // [2][B][kMaxTerms]
    int* cnt = idx + 2 * B * kMaxTerms;                  // [2][B]
    const V* gam = (const V*)Y.gam + (size_t)t.s * Y.gps;
    bool single = true;
    for (int q = lane; q < 2 * B; q += 32) {
        const int side = q / B, rc = q % B;              // side 0: rows at k, side 1: columns at k'
        const int kk = side == 0 ? t.k : t.kp;
        const int v = rc / nc, c = rc % nc, ik = kk * nb;
        const int fv = __ldg(Y.mfirst + ik + v), mv = __ldg(Y.msize + ik + v);
        const int fc = __ldg(Y.mfirst + ik + nv + c) - nv, mc = __ldg(Y.msize + ik + nv + c);
        const int64_t ko = __ldg(Y.koff + kk);
        const V* gv = gam + ko + __ldg(Y.boff + ik + v);
        const V* gc = gam + ko + __ldg(Y.boff + ik + nv + c);
        int n = 0;
        for (int a = 0; a < mv; ++a)
            for (int b = 0; b < mc; ++b) {
                const V hv = gv[a * mv + (v - fv)], hc = gc[b * mc + (c - fc)];
                fac[(side * B + rc) * kMaxTerms + n] = side == 0 ? cmc(hv, hc) : cmc(hc, hv);
                idx[(side * B + rc) * kMaxTerms + n] = (fv + a) * nc + fc + b;
                ++n;
            }
        cnt[side * B + rc] = n;
        single = single && n == 1;
    }
    single = __all_sync(0xffffffffu, single);
    __syncwarp();
    const V* S = X + t.src;
    if (single) {
#pragma unroll 8
        for (int e = lane; e < B * B; e += 32) {
            const int r = e % B, col = e / B;
            const V x = S[(int64_t)idx[(B + col) * kMaxTerms] * t.ld + idx[r * kMaxTerms]];
            V acc = cm(cm(fac[r * kMaxTerms], x), fac[(B + col) * kMaxTerms]);
            X[t.dst + (int64_t)col * t.ld + r] = acc;
            if (t.flags & 1) {
                acc.y = -acc.y;
                X[t.dstm + (int64_t)r * t.ld + col] = acc;
            }
        }
        return;
    }
    for (int e = lane; e < B * B; e += 32) {
        const int r = e % B, col = e / B;
        const int nr = cnt[r], ncl = cnt[B + col];
        V acc;
        acc.x = acc.y = R(0);
        for (int i = 0; i < nr; ++i) {
            const V Lf = fac[r * kMaxTerms + i];
            const int srow = idx[r * kMaxTerms + i];
            for (int j = 0; j < ncl; ++j) {
                const int scol = idx[(B + col) * kMaxTerms + j];
                const V p = cm(cm(Lf, S[(int64_t)scol * t.ld + srow]), fac[(B + col) * kMaxTerms + j]);
                acc.x += p.x;
                acc.y += p.y;
            }
        }
        X[t.dst + (int64_t)col * t.ld + r] = acc;
        if (t.flags & 1) {
            acc.y = -acc.y;
            X[t.dstm + (int64_t)r * t.ld + col] = acc;
        }
    }
}

template <typename R, bool kBatch>
int launch_rotate_t(const RotSys* systems, const RotSys& one, int B, const RotTask* tasks, int64_t n, void* X,
                    cudaStream_t st) {
    using V = typename C2r<R>::T;
    if (n == 0) return BSE_OK;
    const size_t sm = kRotWarps * rot_warp_bytes(B, sizeof(V));
    if (sm > 227 * 1024) return fail(BSE_EUNSUPPORTED, "rotation of %d x %d blocks exceeds shared memory", B, B);
    cudaError_t e = cudaFuncSetAttribute(rotate_kernel<R, kBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "rotate smem: %s", cudaGetErrorString(e));
    const int64_t per_launch = (int64_t)kRotWarps << 30;
    for (int64_t off = 0; off < n; off += per_launch) {
        const int64_t nt = n - off < per_launch ? n - off : per_launch;
        rotate_kernel<R, kBatch><<<(unsigned)((nt + kRotWarps - 1) / kRotWarps), kRotWarps * 32, sm, st>>>(
            systems, one, tasks + off, nt, B, (V*)X);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(BSE_ECUDA, "rotate launch: %s", cudaGetErrorString(e));
    }
    return BSE_OK;
}

}  // namespace

namespace {

__global__ void rot_tasks_kernel(RotTables g, const RotTile* __restrict__ tiles, int ntiles, int64_t npairs,
                                 const int* __restrict__ jr_of, const int* __restrict__ gop_of,
                                 const int* __restrict__ seedpre, RotTask* out, int* status) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    int lo = 0, hi = ntiles - 1;   // the tile of pair p: last one starting at or before p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tiles[mid].pair_off <= p) lo = mid;
        else hi = mid - 1;
    }
    const RotTile T = tiles[lo];
    const int na = g.star_off[T.a + 1] - g.star_off[T.a], nb = g.star_off[T.b + 1] - g.star_off[T.b];
    const int64_t q = p - T.pair_off;
    int i, j;
    if (T.tri) {   // row i holds j = i .. nb-1
        int64_t r = q;
        int len = nb;
        i = 0;
        while (r >= len && i + 1 < na) {
            r -= len;
            ++i;
            --len;
        }
        j = i + (int)r;
    } else {
        i = (int)(q / nb);
        j = (int)(q % nb);
    }
    if (i >= na || j >= nb) {
        atomicOr(status, 2);
        return;
    }
    const int k = g.star_k[g.star_off[T.a] + i], kp = g.star_k[g.star_off[T.b] + j];
    const int k0 = g.star_k[g.star_off[T.a]];
    const int s1 = g.inv[g.s_k[k]];   // takes k to k0
    const int jpp = g.pos_in_star[g.rotk[(int64_t)s1 * g.nk + kp]];
    const int jr = jr_of[T.rep_off + jpp];
    const int s = g.mult[gop_of[T.rep_off + jpp] * g.nops + s1];
    const int r = g.star_k[g.star_off[T.b] + jr];
    if (g.rotk[(int64_t)s * g.nk + k] != k0 || g.rotk[(int64_t)s * g.nk + kp] != r) {
        atomicOr(status, 2);
        return;
    }
    if (i == 0 && j == jr) return;   // a seed: computed by the direct kernel
    const int64_t ridx = i == 0 ? q - seedpre[T.rep_off + j] : q - T.seeds;
    const int64_t B = g.B, rows = T.rows;
    RotTask o;
    o.src = T.xoff + (int64_t)jr * B * rows;
    o.dst = T.xoff + (int64_t)j * B * rows + (int64_t)i * B;
    o.dstm = T.xoff + (int64_t)i * B * rows + (int64_t)j * B;
    o.k = k;
    o.kp = kp;
    o.s = s;
    o.ld = T.rows;
    o.flags = (T.tri && j > i) ? 1 : 0;
    o.pad = 0;
    out[T.rot_off + ridx] = o;
}

}  // namespace

int launch_rot_tasks(const RotTables& g, const RotTile* tiles, int ntiles, int64_t npairs, const int* jr,
                     const int* gop, const int* seedpre, RotTask* out, int* status, cudaStream_t st) {
    if (npairs == 0 || ntiles == 0) return BSE_OK;
    rot_tasks_kernel<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(g, tiles, ntiles, npairs, jr, gop, seedpre,
                                                                         out, status);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

int launch_rotate(const RotSys& one, int prec32, const RotTask* tasks, int64_t n, void* X, cudaStream_t st) {
    return prec32 ? launch_rotate_t<float, false>(nullptr, one, one.nv * one.nc, tasks, n, X, st)
                  : launch_rotate_t<double, false>(nullptr, one, one.nv * one.nc, tasks, n, X, st);
}

int launch_rotate_multi(const RotSys* systems, int bmax, int prec32, const RotTask* tasks, int64_t n, void* X,
                        cudaStream_t st) {
    RotSys none{};
    return prec32 ? launch_rotate_t<float, true>(systems, none, bmax, tasks, n, X, st)
                  : launch_rotate_t<double, true>(systems, none, bmax, tasks, n, X, st);
}

}  // namespace bse
