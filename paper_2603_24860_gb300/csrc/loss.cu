// Longitudinal excitons and the loss spectrum (Sec. III.D, "Excitonic
// energies and loss spectrum"; sm_103a).
//
// The unmodified Coulomb interaction adds alpha B* B^T to H (Eq. epsinv_div;
// alpha = 4 pi spin / N_k with B of Eq. oscillator).  In the eigenbasis of a
// block the new levels are the roots of the secular equation (Eq. secular)
//   f(x) = 1 - alpha sum_l w_l / (x - Omega_l),   w_l = |B_l|^2,
// one in each gap between consecutive levels with w_l > 0 and one above the
// highest; levels with w_l = 0 stay.  The eigenvectors are known in closed
// form (Eq. eigenvec_xi), giving the strength of a longitudinal exciton
// |B'_x|^2 = 1 / (alpha f'(x)) with f'(x) = alpha sum_l w_l / (x - Omega_l)^2.
//
// One warp per root: the lanes share the sum over the levels; the root is
// found on its bracket by Newton steps that fall back to bisection when they
// leave it, in the shifted variable x = Omega_j + delta so that the distance
// to the nearest pole keeps its relative accuracy.
#include <cuda_runtime.h>

#include <cfloat>

#include "fp64_fast.h"
#include "internal.h"

namespace bse {

namespace {

constexpr int kLossThreads = 1024;

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// bright levels (w > rel * max w), in order, and their count and total strength (one block)
__global__ void compact_kernel(const double* __restrict__ Om, const double* __restrict__ osc, int64_t n, double rel,
                               double* ob, double* wb, int* m_out, double* wtot) {
    __shared__ double s_red[kLossThreads / 32];
    __shared__ int s_scan[kLossThreads];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    double mx = 0.0;
    for (int64_t i = tid; i < n; i += blockDim.x) mx = fmax(mx, osc[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_red[wid] = mx;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmax(a, s_red[w]);
        s_red[0] = a;
    }
    __syncthreads();
    const double thr = rel * s_red[0];
    // contiguous chunk per thread, then an exclusive scan of the chunk counts
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t i0 = tid * per, i1 = min(n, i0 + per);
    int cntb = 0;
    for (int64_t i = i0; i < i1; ++i) cntb += osc[i] > thr;
    s_scan[tid] = cntb;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int v = tid >= off ? s_scan[tid - off] : 0;
        __syncthreads();
        s_scan[tid] += v;
        __syncthreads();
    }
    int pos = s_scan[tid] - cntb;
    for (int64_t i = i0; i < i1; ++i)
        if (osc[i] > thr) {
            ob[pos] = Om[i];
            wb[pos] = osc[i];
            ++pos;
        }
    if (tid == blockDim.x - 1) *m_out = s_scan[tid];
    __syncthreads();
    // total strength (fixed order)
    double s = 0.0;
    const int m = s_scan[blockDim.x - 1];
    for (int i = tid; i < m; i += blockDim.x) s += wb[i];
    s = wsum(s);
    if (lane == 0) s_red[wid] = s;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += s_red[w];
        *wtot = a;
    }
}

// f(delta) and f'(delta) for the root above level j (warp-wide sums)
__device__ __forceinline__ void secular_eval(const double* __restrict__ ob, const double* __restrict__ wb, int m, int j,
                                             double delta, double alpha, int lane, double& f, double& fp) {
    double s1 = 0.0, s2 = 0.0;
    const double oj = ob[j];
    for (int l = lane; l < m; l += 32) {
        const double den = (oj - ob[l]) + delta;
        const double r = rcp_nr(den);
        const double t = wb[l] * r;
        s1 += t;
        s2 = fma(t, r, s2);
    }
    s1 = wsum(s1);
    s2 = wsum(s2);
    f = 1.0 - alpha * s1;
    fp = alpha * s2;
}

__global__ void secular_kernel(const double* __restrict__ ob, const double* __restrict__ wb, const int* __restrict__ m_ptr,
                               const double* __restrict__ wtot, double alpha, double* root, double* str) {
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int m = *m_ptr;
    if (j >= m) return;
    const double lo = ob[j];
    const double hi = j + 1 < m ? ob[j + 1] : ob[j] + alpha * *wtot;
    const double gap = hi - lo;
    if (!(gap > 0.0)) {   // a level repeated exactly: the root sits on it with no strength
        if (lane == 0) {
            root[j] = lo;
            str[j] = 0.0;
        }
        return;
    }
    double a = 0.0, b = gap, d = 0.5 * gap, f = 0.0, fp = 1.0;
    for (int it = 0; it < 200; ++it) {
        secular_eval(ob, wb, m, j, d, alpha, lane, f, fp);
        if (f < 0.0) a = d;
        else b = d;
        double dn = d - f / fp;
        if (!(dn > a && dn < b)) dn = 0.5 * (a + b);
        // relative to delta itself: delta is held exactly, so a root next to its
        // pole (a nearly dark level, delta ~ alpha w_j) keeps its accuracy
        if (fabs(dn - d) <= 4.0 * DBL_EPSILON * dn || b - a <= 4.0 * DBL_EPSILON * b) {
            d = dn;
            break;
        }
        d = dn;
    }
    secular_eval(ob, wb, m, j, d, alpha, lane, f, fp);
    if (lane == 0) {
        root[j] = lo + d;
        str[j] = (fp > 0.0 && fp < DBL_MAX) ? 1.0 / (alpha * fp) : 0.0;
    }
}

// all n levels in ascending order: the m roots with their strengths and the
// n - m levels that kept w <= threshold (strength 0); ties by origin
__global__ void loss_rank_kernel(const double* __restrict__ Om, const double* __restrict__ osc, int64_t n, double rel,
                                 const double* __restrict__ root, const double* __restrict__ str,
                                 const int* __restrict__ m_ptr, double* out_l, double* out_w) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int m = *m_ptr;
    // element t: root t for t < m, else the (t - m)-th dark level
    double mx = 0.0;
    for (int64_t i = 0; i < n; ++i) mx = fmax(mx, __ldg(osc + i));
    const double thr = rel * mx;
    double x, w;
    if (t < m) {
        x = root[t];
        w = str[t];
    } else {
        int64_t c = -1, i = 0;
        for (; i < n; ++i)
            if (!(__ldg(osc + i) > thr) && ++c == t - m) break;
        if (i >= n) return;   // cannot happen: n - m levels are below the threshold
        x = Om[i];
        w = 0.0;
    }
    int64_t pos = 0;
    for (int64_t u = 0; u < m; ++u) {
        const double y = root[u];
        pos += (y < x) || (y == x && u < t);
    }
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (__ldg(osc + i) > thr) continue;
        const double y = Om[i];
        const int64_t u = m + c;
        pos += (y < x) || (y == x && u < t);
        ++c;
    }
    out_l[pos] = x;
    out_w[pos] = w;
}

}  // namespace

size_t loss_scratch_bytes(int64_t n) { return sizeof(double) * (size_t)(4 * n + 8) + 256; }

int launch_loss_levels(const double* Om, const double* osc, int64_t n, double alpha, void* scratch, double* out_l,
                       double* out_w, cudaStream_t st) {
    if (n < 1) return BSE_OK;
    const double rel = 1e-14;
    double* ob = (double*)scratch;
    double* wb = ob + n;
    double* root = wb + n;
    double* str = root + n;
    double* wtot = str + n;
    int* m = (int*)(wtot + 2);
    compact_kernel<<<1, kLossThreads, 0, st>>>(Om, osc, n, rel, ob, wb, m, wtot);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    secular_kernel<<<(unsigned)((32 * n + 255) / 256), 256, 0, st>>>(ob, wb, m, wtot, alpha, root, str);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    loss_rank_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Om, osc, n, rel, root, str, m, out_l, out_w);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

}  // namespace bse
