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

// One thread per element of a rotated block (slots of bsq = B_max^2 per
// task): out[(v c),(v' c')] = sum over the multiplets of v, c at k and of
// v', c' at k' of conj(Gamma_c(k)[c1][c]) Gamma_v(k)[v1][v] S[(v1 c1),(v2 c2)]
// Gamma_c(k')[c2][c'] conj(Gamma_v(k')[v2][v']) -- one term when the four
// multiplets are single bands (every k of a general star), at most 81.
template <typename R, bool kBatch>
__global__ void __launch_bounds__(256) rotate_kernel(const RotSys* __restrict__ systems,
                                                     const __grid_constant__ RotSys one,
                                                     const RotTask* __restrict__ tasks, int64_t ntasks, int bsq,
                                                     typename C2r<R>::T* X) {
    using V = typename C2r<R>::T;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ti = g / bsq;
    if (ti >= ntasks) return;
    const int e = (int)(g - ti * bsq);
    const RotTask& t = tasks[ti];
    const RotSys& Y = kBatch ? systems[t.flags >> 1] : one;
    const int nv = Y.nv, nc = Y.nc, nb = Y.nb, B = nv * nc;
    if (e >= B * B) return;
    const int r = e % B, col = e / B;
    const int v = r / nc, c = r % nc, vp = col / nc, cp = col % nc;
    const int k = t.k, kp = t.kp;
    const V* gam = (const V*)Y.gam + (size_t)t.s * Y.gps;
    const int ik = k * nb, ikp = kp * nb;
    const int fv = __ldg(Y.mfirst + ik + v), mv = __ldg(Y.msize + ik + v);
    const int fc = __ldg(Y.mfirst + ik + nv + c) - nv, mc = __ldg(Y.msize + ik + nv + c);
    const int fvp = __ldg(Y.mfirst + ikp + vp), mvp = __ldg(Y.msize + ikp + vp);
    const int fcp = __ldg(Y.mfirst + ikp + nv + cp) - nv, mcp = __ldg(Y.msize + ikp + nv + cp);
    const V* gvk = gam + __ldg(Y.koff + k) + __ldg(Y.boff + ik + v);
    const V* gck = gam + __ldg(Y.koff + k) + __ldg(Y.boff + ik + nv + c);
    const V* gvp = gam + __ldg(Y.koff + kp) + __ldg(Y.boff + ikp + vp);
    const V* gcp = gam + __ldg(Y.koff + kp) + __ldg(Y.boff + ikp + nv + cp);
    V acc;
    acc.x = acc.y = R(0);
    for (int a = 0; a < mv; ++a) {
        const V g2 = gvk[a * mv + (v - fv)];
        for (int b = 0; b < mc; ++b) {
            const V L = cmc(g2, gck[b * mc + (c - fc)]);          // Gamma_v(k)[v1][v] conj(Gamma_c(k)[c1][c])
            const int row = (fv + a) * nc + fc + b;
            for (int a2 = 0; a2 < mvp; ++a2) {
                const V h2 = gvp[a2 * mvp + (vp - fvp)];
                for (int b2 = 0; b2 < mcp; ++b2) {
                    const V Rt = cmc(gcp[b2 * mcp + (cp - fcp)], h2);   // Gamma_c(k')[c2][c'] conj(Gamma_v(k')[v2][v'])
                    const V sv = X[t.src + (int64_t)((fvp + a2) * nc + fcp + b2) * t.ld + row];
                    const V p = cm(cm(L, sv), Rt);
                    acc.x += p.x;
                    acc.y += p.y;
                }
            }
        }
    }
    X[t.dst + (int64_t)col * t.ld + r] = acc;
    if (t.flags & 1) {
        acc.y = -acc.y;
        X[t.dstm + (int64_t)r * t.ld + col] = acc;
    }
}

template <typename R, bool kBatch>
int launch_rotate_t(const RotSys* systems, const RotSys& one, int B, const RotTask* tasks, int64_t n, void* X,
                    cudaStream_t st) {
    using V = typename C2r<R>::T;
    if (n == 0) return BSE_OK;
    const int bsq = B * B;
    const int64_t per = ((int64_t)1 << 31) / bsq;   // tasks per launch: at most 2^31 threads
    for (int64_t off = 0; off < n; off += per) {
        const int64_t nt = n - off < per ? n - off : per;
        const int64_t threads = nt * bsq;
        rotate_kernel<R, kBatch><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(systems, one, tasks + off, nt,
                                                                                 bsq, (V*)X);
        note_launch();
        cudaError_t e = cudaGetLastError();
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
