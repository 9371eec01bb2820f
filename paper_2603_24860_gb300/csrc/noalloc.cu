// Head correction W^div computed without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need
// this value: frameworks that own the whole device memory budget through
// their own pool and must account for every byte, latency-critical loops in
// which the implicit device synchronisation of cudaMalloc / cudaFree is not
// acceptable, and plug-ins that are handed only pre-allocated buffers.  This
// entry point serves them: the block partial sums of the lattice sum live in
// a fixed array in the library's own device memory, the caller passes the
// output buffer, and nothing is allocated (no cudaMalloc, no cudaFree, no
// allocating library routine).
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "internal.h"

namespace bse {
double head_h00(const double* L);
}

using namespace bse;

// Maximum number of block partial sums of the lattice sum (256 Q columns per
// block).  65536 doubles = 512 KiB, resident on every device that loads the
// library until the process exits.
#define BSE_NOALLOC_MAX_PARTIALS 65536
// Longest lattice column one thread sums (points along the third axis); far
// above what any mesh within the partial-sum limit needs
#define BSE_NOALLOC_MAX_COLUMN 65536

static __device__ __align__(256) double g_noalloc_partials[BSE_NOALLOC_MAX_PARTIALS];

// Host-side address of g_noalloc_partials on each device, looked up once per
// device (the symbol's name is only a host stand-in, not a device address).
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {};

static int noalloc_scratch(double** out) {
    int dev = -1;
    BSE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(BSE_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess)
            return fail(BSE_ECUDA, "cudaGetSymbolAddress of the fixed scratch: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<double*>(g_noalloc_ptr[dev]);
    return BSE_OK;
}

// w = c0 - c1 * w with both operations rounded separately.  The result agrees
// with the W^div of bse_create to about 1e-10 relative, not bit for bit:
// bse_create sums one point per orbit of the point group (weighted by the
// orbit size) and may round its last step differently.
__global__ void noalloc_finalize_kernel(double* w, double c0, double c1) { w[0] = __dsub_rn(c0, __dmul_rn(c1, w[0])); }

extern "C" int bse_head_correction_noalloc(const double* lattice, const int32_t* mesh, const double* eps_inf,
                                           double* w_div_dev, void* stream) {
    clear_error();
    if (!lattice || !mesh || !eps_inf || !w_div_dev) return fail(BSE_EINVAL, "null argument");
    if (mesh[0] <= 0 || mesh[1] <= 0 || mesh[2] <= 0) return fail(BSE_EINVAL, "mesh dimensions must be positive");
    const double* L = lattice;
    double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                 L[2] * (L[3] * L[7] - L[4] * L[6]);
    if (!(std::fabs(det) > 0)) return fail(BSE_EINVAL, "lattice is singular");
    // reciprocal basis b_j = 2 pi (L^{-T})_{:, j}, row-major with columns b_j
    double inv[9] = {(L[4] * L[8] - L[5] * L[7]) / det, (L[2] * L[7] - L[1] * L[8]) / det,
                     (L[1] * L[5] - L[2] * L[4]) / det, (L[5] * L[6] - L[3] * L[8]) / det,
                     (L[0] * L[8] - L[2] * L[6]) / det, (L[2] * L[3] - L[0] * L[5]) / det,
                     (L[3] * L[7] - L[4] * L[6]) / det, (L[1] * L[6] - L[0] * L[7]) / det,
                     (L[0] * L[4] - L[1] * L[3]) / det};
    double rl[18];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) rl[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
    for (int i = 0; i < 9; ++i) rl[9 + i] = L[i];
    const int n[3] = {mesh[0], mesh[1], mesh[2]};
    const double v_uc = std::fabs(det);
    const int64_t nk = (int64_t)n[0] * n[1] * n[2];
    if (nk > INT32_MAX) return fail(BSE_EINVAL, "mesh has %lld points, more than 2^31 - 1", (long long)nk);
    const double b = 0.005;
    const double qmax = std::sqrt(-std::log(b) / b);
    const double delta = std::cbrt(8.0 * M_PI * M_PI * M_PI / v_uc / (double)nk);
    const int64_t need = wdiv_partials(L, n, qmax, delta);
    if (need > BSE_NOALLOC_MAX_PARTIALS)
        return fail(BSE_EINVAL, "mesh too fine for the fixed scratch: the lattice sum needs %lld partial sums, "
                    "at most %d are available", (long long)need, BSE_NOALLOC_MAX_PARTIALS);
    const int64_t col = wdiv_column_length(L, n, qmax, delta);
    if (col > BSE_NOALLOC_MAX_COLUMN)
        return fail(BSE_EINVAL, "mesh too fine along its third axis: a lattice column has %lld points, at most %d",
                    (long long)col, BSE_NOALLOC_MAX_COLUMN);
    double* scratch = nullptr;
    BSE_TRY(noalloc_scratch(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    // every partial that the reduction reads is written first by the lattice-sum
    // kernel of this call, so no part of the scratch has to start at zero
    BSE_TRY(launch_wdiv(rl, n, eps_inf, b, qmax, delta, scratch, BSE_NOALLOC_MAX_PARTIALS, w_div_dev, st));
    const double integral = M_PI * head_h00(eps_inf) / std::sqrt(b) * std::erf(std::sqrt(b) * qmax);
    noalloc_finalize_kernel<<<1, 1, 0, st>>>(w_div_dev, integral / (2.0 * M_PI * M_PI),
                                             4.0 * M_PI / ((double)nk * v_uc));
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}
