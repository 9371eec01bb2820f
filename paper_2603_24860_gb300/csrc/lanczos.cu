// Lanczos-Haydock spectrum of a block (Sec. IV: the spectrum without the
// diagonalisation, summed over the contributing blocks) on sm_103a.
//
// The Hermitian Lanczos recurrence from the dipole direction c = conj(b)
// (b = U^T B, whose spectral measure gives |B_lambda|^2, Eq. oscillatorA),
// without reorthogonalisation:
//   w = H v_j - beta_j v_{j-1},  alpha_j = Re <v_j, w>,  u_{j+1} = w - alpha_j v_j,
//   beta_{j+1} = |u_{j+1}|,  v_{j+1} = u_{j+1} / beta_{j+1}.
// The vectors are kept unnormalised (u_j = beta_j v_j, three rotating
// buffers), so a step needs two grid-wide sums and two grid barriers.  The
// tridiagonal T_m = (alpha, beta) then gives the Ritz values and Gauss
// weights (levels of T_m and |c|^2 times the squared first components) whose
// Lorentzian sum is the continued fraction of the Haydock method.  Im eps is
// evaluated from the fraction itself (one thread per frequency); when the
// Ritz pairs are asked for, T_m (small, and without reorthogonalisation with
// near-coincident Ritz values, copies of converged ones) goes to a dense
// symmetric eigensolver, for which such clusters are harmless.
//
// GB300 layout: one persistent cooperative kernel, one CTA per SM.  Every CTA
// holds v_j in shared memory; (H v)_r is the dot product of column r with v
// (H is Hermitian: (H v)_r = sum_i conj(H_ir) v_i), one warp per column, so
// the block is read once per step with coalesced loads and no cross-CTA
// reduction except the two scalars.  The FP64 pipe bounds a step: 4 n^2 DFMA
// plus one shuffle reduction per column.  One FP64 warp instruction occupies
// its sub-partition's pipe for 64 cycles whatever its active lanes, so a
// column is not split across warps: the extra reductions would cost more
// than the idle SMs of small blocks (n < 8 x 152).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fp64_fast.h"
#include "grid_sync.h"
#include "internal.h"

namespace bse {

namespace {

constexpr int kLzThreads = 256;
constexpr int kLzWarps = kLzThreads / 32;

__device__ __forceinline__ double lz_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// u_0 = conj(b), beta_0 = |b| (one block)
__global__ void lanczos_start_kernel(const double2* __restrict__ b, int64_t n, double2* u0, double* beta) {
    __shared__ double s[kLzWarps];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 x = b[i];
        u0[i] = make_double2(x.x, -x.y);
        acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    acc = lz_warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        beta[0] = sqrt(t);
    }
}

struct LzArgs {
    const double2* H;   // n x n column-major, leading dimension ld (read only)
    int64_t ld, n;
    int m;              // steps requested
    double2* U;         // [3][n] unnormalised Lanczos vectors, u_0 = c on entry
    double* part1;      // [G] per-CTA parts of Re <v_j, w>
    double* part2;      // [G] per-CTA parts of |u_{j+1}|^2
    double* alpha;      // [m]
    double* beta;       // [m + 1], beta[0] = |c| on entry
    int* done;          // steps performed
    unsigned* bar;      // barrier counter, zero on entry
    int* err;           // error flag, zero on entry
    long spin;          // polls of a grid barrier before it gives up
};

__global__ void __launch_bounds__(kLzThreads, 1) lanczos_kernel(LzArgs a) {
    extern __shared__ __align__(16) double2 s_v[];   // v_j
    __shared__ double s_red[kLzWarps];
    __shared__ double s_tot;
    __shared__ int s_flag;
    const int n = (int)a.n, G = gridDim.x, blk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gw = blk * kLzWarps + wid, nw = G * kLzWarps;
    unsigned nbar = 0;
    double bj = __ldcg(a.beta), bjm1 = 1.0;
    int steps = a.m;

    // this CTA's part of a sum (tid 0 writes it; the grid barrier that follows orders the write)
    auto block_part = [&](double v, double* part) {
        v = lz_warp_sum(v);
        if (lane == 0) s_red[wid] = v;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kLzWarps; ++w) t += s_red[w];
            part[blk] = t;
        }
    };
    // the sum of all parts, in the same order in every CTA
    auto grid_total = [&](const double* part) -> double {
        if (wid == 0) {
            double v = 0.0;
            for (int b = lane; b < G; b += 32) v += __ldcg(part + b);
            v = lz_warp_sum(v);
            if (lane == 0) s_tot = v;
        }
        __syncthreads();
        const double t = s_tot;
        __syncthreads();
        return t;
    };

    for (int j = 0; j < a.m; ++j) {
        const double2* uj = a.U + (size_t)(j % 3) * n;
        const double2* ujm1 = a.U + (size_t)((j + 2) % 3) * n;
        double2* ujp1 = a.U + (size_t)((j + 1) % 3) * n;
        const double inv = 1.0 / bj;
        for (int i = tid; i < n; i += kLzThreads) {
            const double2 u = __ldcg(uj + i);
            s_v[i] = make_double2(u.x * inv, u.y * inv);
        }
        __syncthreads();
        // y = H v_j - beta_j v_{j-1} on own columns (v_{j-1} = u_{j-1} / beta_{j-1})
        const double cprev = j > 0 ? bj / bjm1 : 0.0;
        double p1 = 0.0;
        for (int r = gw; r < n; r += nw) {
            const double2* col = a.H + (size_t)r * a.ld;
            double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
            int i = lane;
            for (; i + 32 < n; i += 64) {
                const double2 h0 = __ldg(col + i), v0 = s_v[i], h1 = __ldg(col + i + 32), v1 = s_v[i + 32];
                ax = fma(h0.x, v0.x, fma(h0.y, v0.y, ax));
                ay = fma(h0.x, v0.y, fma(-h0.y, v0.x, ay));
                bx = fma(h1.x, v1.x, fma(h1.y, v1.y, bx));
                by = fma(h1.x, v1.y, fma(-h1.y, v1.x, by));
            }
            if (i < n) {
                const double2 h0 = __ldg(col + i), v0 = s_v[i];
                ax = fma(h0.x, v0.x, fma(h0.y, v0.y, ax));
                ay = fma(h0.x, v0.y, fma(-h0.y, v0.x, ay));
            }
            const double sx = lz_warp_sum(ax + bx), sy = lz_warp_sum(ay + by);
            if (lane == 0) {
                double2 y = make_double2(sx, sy);
                if (j > 0) {
                    const double2 q = __ldcg(ujm1 + r);
                    y.x = fma(-cprev, q.x, y.x);
                    y.y = fma(-cprev, q.y, y.y);
                }
                ujp1[r] = y;
                const double2 v = s_v[r];
                p1 = fma(v.x, y.x, fma(v.y, y.y, p1));   // Re(conj(v) y)
            }
        }
        block_part(p1, a.part1);
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;
        const double al = grid_total(a.part1);
        // u_{j+1} = y - alpha_j v_j on own columns (the thread that wrote y)
        double p2 = 0.0;
        if (lane == 0)
            for (int r = gw; r < n; r += nw) {
                double2 y = __ldcg(ujp1 + r);
                const double2 v = s_v[r];
                y.x = fma(-al, v.x, y.x);
                y.y = fma(-al, v.y, y.y);
                ujp1[r] = y;
                p2 = fma(y.x, y.x, fma(y.y, y.y, p2));
            }
        block_part(p2, a.part2);
        if (!grid_barrier(a.bar, (++nbar) * G, a.err, &s_flag, a.spin)) return;
        const double bn = sqrt(grid_total(a.part2));
        if (blk == 0 && tid == 0) {
            a.alpha[j] = al;
            a.beta[j + 1] = bn;
        }
        if (!(bn > 1e-14 * (fabs(al) + bj))) {   // an invariant subspace: T_{j+1} is exact (same in every CTA)
            steps = j + 1;
            break;
        }
        bjm1 = bj;
        bj = bn;
    }
    if (blk == 0 && tid == 0) *a.done = steps;
}

// T_m as a dense k x k column-major matrix: alpha on the diagonal, beta1[j] coupling j and j + 1
__global__ void tm_dense_kernel(const double* __restrict__ alpha, const double* __restrict__ beta1, int k, double* T) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)k * k) return;
    const int r = (int)(id % k), c = (int)(id / k);
    T[id] = r == c ? alpha[r] : (r == c + 1 ? beta1[c] : (c == r + 1 ? beta1[r] : 0.0));
}

// Gauss weights scale z_0(j)^2 from the eigenvector matrix (column j = eigenvector j)
__global__ void tm_weights_kernel(const double* __restrict__ V, int k, double scale, double* w) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const double z = V[(size_t)j * k];
    w[j] = scale * z * z;
}

// Im eps_M(omega) = pref (-Im g(omega + i eta) + Im g(-omega + i eta)) with the continued fraction
// g(z) = norm2 / (z - a_0 - b_1^2 / (z - a_1 - ... / (z - a_{k-1}))) evaluated from the bottom up;
// beta1[j] couples j and j + 1.  Every denominator has imaginary part >= eta > 0.
__global__ void cf_spectrum_kernel(const double* __restrict__ alpha, const double* __restrict__ beta1, int k,
                                   double norm2, const double* __restrict__ omega, int64_t n_omega, double eta,
                                   double pref, double* im) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_omega) return;
    auto im_g = [&](double x) -> double {
        double tr = x - alpha[k - 1], ti = eta;
        for (int j = k - 2; j >= 0; --j) {
            const double b = beta1[j];
            const double r = b * b * rcp_nr(fma(tr, tr, ti * ti));   // b^2 / t = r conj(t)
            tr = fma(-r, tr, x - alpha[j]);
            ti = fma(r, ti, eta);
        }
        return -norm2 * ti * rcp_nr(fma(tr, tr, ti * ti));
    };
    const double w = omega[i];
    im[i] = pref * (im_g(-w) - im_g(w));
}

}  // namespace

int launch_cf_spectrum(const double* alpha, const double* beta1, int k, double norm2, const double* omega,
                       int64_t n_omega, double eta, double pref, double* im, cudaStream_t st) {
    if (n_omega < 1) return BSE_OK;
    cf_spectrum_kernel<<<(unsigned)((n_omega + 127) / 128), 128, 0, st>>>(alpha, beta1, k, norm2, omega, n_omega,
                                                                            eta, pref, im);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

int launch_tm_dense(const double* alpha, const double* beta1, int k, double* T, cudaStream_t st) {
    tm_dense_kernel<<<(unsigned)(((int64_t)k * k + 255) / 256), 256, 0, st>>>(alpha, beta1, k, T);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

int launch_tm_weights(const double* V, int k, double scale, double* w, cudaStream_t st) {
    tm_weights_kernel<<<(unsigned)((k + 255) / 256), 256, 0, st>>>(V, k, scale, w);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

int lanczos_max_dim() { return 12000; }   // v_j in shared memory (192 KB)

size_t lanczos_scratch_bytes(int64_t n, int m) {
    return sizeof(double2) * (size_t)(3 * n) + sizeof(double) * (size_t)(2 * 1024 + 2 * m + 1) + 6 * 256 + 64;
}

int launch_lanczos(const double2* h, int64_t ld, int64_t n, const double2* b, int steps, void* scratch,
                   double** alpha, double** beta, int* done, cudaStream_t st, long wait_polls) {
    if (n < 1 || n > lanczos_max_dim())
        return fail(BSE_EUNSUPPORTED, "Lanczos path: block dimension %lld (at most %d)", (long long)n, lanczos_max_dim());
    if (steps < 1) return fail(BSE_EINVAL, "Lanczos path: %d steps", steps);
    char* p = (char*)scratch;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)q;
    };
    double2* U = (double2*)take(sizeof(double2) * 3 * n);
    double* part1 = (double*)take(sizeof(double) * 1024);
    double* part2 = (double*)take(sizeof(double) * 1024);
    double* al = (double*)take(sizeof(double) * steps);
    double* be = (double*)take(sizeof(double) * (steps + 1));
    int* dn = (int*)take(sizeof(int));
    unsigned* bar = (unsigned*)take(sizeof(unsigned));
    int* err = (int*)take(sizeof(int));

    int dev = 0, sms = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int G = (int)std::min<int64_t>(std::min(sms, 1024), std::max<int64_t>(1, (n + kLzWarps - 1) / kLzWarps));
    const size_t dyn = sizeof(double2) * (size_t)n;
    BSE_CUDA(cudaFuncSetAttribute(lanczos_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lanczos_kernel, kLzThreads, dyn));
    if (per_sm < 1 || G > per_sm * sms) return fail(BSE_EUNSUPPORTED, "Lanczos kernel cannot be co-resident");

    BSE_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned), st));
    BSE_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    lanczos_start_kernel<<<1, kLzThreads, 0, st>>>(b, n, U, be);
    note_launch();
    BSE_CUDA(cudaGetLastError());
    LzArgs a;
    a.H = h;
    a.ld = ld;
    a.n = n;
    a.m = steps;
    a.U = U;
    a.part1 = part1;
    a.part2 = part2;
    a.alpha = al;
    a.beta = be;
    a.done = dn;
    a.bar = bar;
    a.err = err;
    a.spin = wait_limit(wait_polls, kGridSpinLimit);
    void* args[] = {&a};
    BSE_CUDA(cudaLaunchCooperativeKernel((const void*)lanczos_kernel, dim3(G), dim3(kLzThreads), args, dyn, st));
    note_launch();
    int hv[2] = {0, 0};
    BSE_CUDA(cudaMemcpyAsync(&hv[0], dn, sizeof(int), cudaMemcpyDeviceToHost, st));
    BSE_CUDA(cudaMemcpyAsync(&hv[1], err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BSE_CUDA(cudaStreamSynchronize(st));
    if (hv[1]) return fail(BSE_ETIMEOUT, "a grid barrier of the Lanczos kernel gave up");
    *alpha = al;
    *beta = be;
    *done = hv[0];
    return BSE_OK;
}

}  // namespace bse
