// Rotated direct-term blocks (Eq. Wtrafo, Sec. III.C.6): the direct term of a
// k pair (k, k') follows from the one of the symmetry-equivalent seed pair
// (s k, s k') by band rotations, since Gamma~(s) commutes with K^d:
//
//   K^d(k, k') = G(s,k)^dagger K^d(sk, sk') G(s,k'),
//   G(s,k)[(v1,c1),(v,c)] = Gamma(s)_{kc}^{sk c1} conj(Gamma(s)_{kv}^{sk v1})   (Eq. Ttilde)
//
// with Gamma(s) block-diagonal over the degenerate multiplets (Eq. Ts), so
// each element is a sum over at most 3 x 3 terms on either side.  One CTA
// per rotated pair: the seed block (already in the tile arena) is staged in
// shared memory, rotated on the right (k') and then on the left (k), and
// written to its place in the tile (with its conjugate transpose when the
// tile is a diagonal star pair).
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

template <typename R, bool kBatch>
__global__ void __launch_bounds__(128) rotate_kernel(const RotSys* __restrict__ systems, const __grid_constant__ RotSys one,
                                                     const RotTask* __restrict__ tasks, typename C2r<R>::T* X) {
    using V = typename C2r<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RotTask t = tasks[blockIdx.x];
    const RotSys& Y = kBatch ? systems[t.flags >> 1] : one;
    const int nv = Y.nv, nc = Y.nc, nb = Y.nb, B = nv * nc;
    V* S = (V*)smem_raw;          // seed block, column-major B x B
    V* T = S + B * B;             // after the right rotation
    const V* gam = (const V*)Y.gam + (size_t)t.s * Y.gps;
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
        const int r = e % B, col = e / B;
        S[e] = X[t.src + (int64_t)col * t.ld + r];
    }
    __syncthreads();
    // right: T[(v1 c1), (v' c')] = sum_{v2 ~ v', c2 ~ c'} S[(v1 c1), (v2 c2)] Gamma_c(k')[c2][c'] conj(Gamma_v(k')[v2][v'])
    {
        const int kp = t.kp;
        const V* gk = gam + Y.koff[kp];
        for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
            const int row = e % B, col = e / B;
            const int vp = col / nc, cp = col % nc;
            const int fv = Y.mfirst[kp * nb + vp], mv = Y.msize[kp * nb + vp];
            const int fc = Y.mfirst[kp * nb + nv + cp] - nv, mc = Y.msize[kp * nb + nv + cp];
            const V* gv = gk + Y.boff[kp * nb + vp];
            const V* gc = gk + Y.boff[kp * nb + nv + cp];
            V acc;
            acc.x = acc.y = R(0);
            for (int a = 0; a < mv; ++a) {
                const V g2 = gv[a * mv + (vp - fv)];
                for (int b = 0; b < mc; ++b) {
                    const V g1 = gc[b * mc + (cp - fc)];
                    const V sv = S[row + ((fv + a) * nc + fc + b) * B];
                    const V p = cmc(cm(sv, g1), g2);
                    acc.x += p.x;
                    acc.y += p.y;
                }
            }
            T[e] = acc;
        }
    }
    __syncthreads();
    // left: out[(v c), (v' c')] = sum_{v1 ~ v, c1 ~ c} conj(Gamma_c(k)[c1][c]) Gamma_v(k)[v1][v] T[(v1 c1), (v' c')]
    {
        const int k = t.k;
        const V* gk = gam + Y.koff[k];
        for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
            const int r = e % B, col = e / B;
            const int v = r / nc, c = r % nc;
            const int fv = Y.mfirst[k * nb + v], mv = Y.msize[k * nb + v];
            const int fc = Y.mfirst[k * nb + nv + c] - nv, mc = Y.msize[k * nb + nv + c];
            const V* gv = gk + Y.boff[k * nb + v];
            const V* gc = gk + Y.boff[k * nb + nv + c];
            V acc;
            acc.x = acc.y = R(0);
            for (int a = 0; a < mv; ++a) {
                const V g2 = gv[a * mv + (v - fv)];
                for (int b = 0; b < mc; ++b) {
                    const V g1 = gc[b * mc + (c - fc)];
                    const V tv = T[((fv + a) * nc + fc + b) + col * B];
                    const V p = cm(cmc(tv, g1), g2);
                    acc.x += p.x;
                    acc.y += p.y;
                }
            }
            X[t.dst + (int64_t)col * t.ld + r] = acc;
            if (t.flags & 1) {
                V m = acc;
                m.y = -m.y;
                X[t.dstm + (int64_t)r * t.ld + col] = m;
            }
        }
    }
}

template <typename R, bool kBatch>
int launch_rotate_t(const RotSys* systems, const RotSys& one, int B, const RotTask* tasks, int64_t n, void* X,
                    cudaStream_t st) {
    using V = typename C2r<R>::T;
    if (n == 0) return BSE_OK;
    const size_t sm = 2 * sizeof(V) * (size_t)B * B;
    if (sm > 227 * 1024) return fail(BSE_EUNSUPPORTED, "rotation of %d x %d blocks exceeds shared memory", B, B);
    cudaError_t e = cudaFuncSetAttribute(rotate_kernel<R, kBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return fail(BSE_ECUDA, "rotate smem: %s", cudaGetErrorString(e));
    for (int64_t off = 0; off < n; off += 1 << 30) {
        const int64_t nt = n - off < (1 << 30) ? n - off : (1 << 30);
        rotate_kernel<R, kBatch><<<(unsigned)nt, 128, sm, st>>>(systems, one, tasks + off, (V*)X);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(BSE_ECUDA, "rotate launch: %s", cudaGetErrorString(e));
    }
    return BSE_OK;
}

}  // namespace

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
