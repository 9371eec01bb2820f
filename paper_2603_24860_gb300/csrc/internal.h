// Internal declarations of the GB300 BSE block builder (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "bse.h"

namespace bse {

using cplx = std::complex<double>;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int fail(int code, const char* fmt, ...);   // records the message, returns code
void clear_error();

#define BSE_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess)                                                 \
            return ::bse::fail(BSE_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__,  \
                               #call, cudaGetErrorString(e_));                 \
    } while (0)

#define BSE_TRY(call)                                                          \
    do {                                                                       \
        int r_ = (call);                                                       \
        if (r_ != BSE_OK) return r_;                                           \
    } while (0)

// ---------------------------------------------------------------------------
// host symmetry tables (host_tables.cpp)
// ---------------------------------------------------------------------------
struct Tables {
    int nops = 0, nk = 0, nv = 0, nc = 0, nb = 0, B = 0;  // B = nv * nc
    int n[3] = {0, 0, 0};
    int64_t N = 0;
    double lattice[9];      // row-major, columns a_j
    double recip[9];        // row-major, columns b_j = 2 pi L^{-T}
    double v_uc = 0.0;
    std::vector<int32_t> rot, rk;     // [nops*9] R and R^{-T}
    std::vector<double> tau;          // [nops*3]
    std::vector<double> cart;         // [nops*9] A = L R L^{-1}
    std::vector<int32_t> mult;        // [nops*nops]
    int identity = -1;
    std::vector<int32_t> kidx;        // [nk*3] mesh indices i, j, l
    std::vector<int32_t> rotk;        // [nops*nk]
    std::vector<int32_t> fold;        // [nops*nk*3] G-bar = R^{-T} f_k - f_{sk}, integer
    std::vector<int32_t> star_of, star_rep, s_k, pos_in_star;
    std::vector<std::vector<int32_t>> stars;
    std::vector<int32_t> class_of;
    int n_irreps = 0;
    std::vector<int32_t> chi, irrep_dim, bright;   // chi [n_irreps*nops]
    // multiplets at each k: (first band, size) for occupied and unoccupied
    std::vector<std::vector<std::pair<int, int>>> vmult, cmult;
    std::vector<int32_t> band_mult;   // [nk*nb] multiplet id of each band (per k)
    int band_mult_size(int k, int band) const {   // size of the band's multiplet at k
        for (auto* ms : {&vmult[k], &cmult[k]})
            for (auto& m : *ms)
                if (band >= m.first && band < m.first + m.second) return m.second;
        return 1;
    }
    // orbits of the product basis
    std::vector<int64_t> orbit_off;     // [n_orbits+1] into orbit_members
    std::vector<int64_t> orbit_members; // product indices, ascending per orbit
    std::vector<int32_t> orbit_star;    // [n_orbits]
    std::vector<int32_t> orbit_vlo, orbit_vn, orbit_clo, orbit_cn;
    std::vector<int32_t> orbit_of;      // [N]
    // band rotations Gamma(s): multiplet blocks, layout below
    std::vector<int64_t> gam_koff;      // [nk+1] entry offset of k within one s
    std::vector<int64_t> gam_boff;      // [nk*nb] offset of the band's multiplet block from gam_koff[k]
    int64_t gam_per_s = 0;              // entries per operation
    std::vector<cplx> gamma;            // [nops * gam_per_s]
};

int build_group(Tables& t, const bse_system* sys);
int build_mesh(Tables& t);
int build_characters(Tables& t);
int build_multiplets_and_orbits(Tables& t, const double* eps_host);
int check_band_rotations(const Tables& t);
// f(0), ..., f(n-1) on the persistent host thread pool (largest cost first when
// costs are given); returns when all have run
void host_parallel_for(int n, const std::function<void(int)>& f, const std::vector<double>* cost = nullptr);

// canonical basis of one irrep (host_tables.cpp)
struct Basis {
    int64_t dim = 0;
    std::vector<int32_t> col_orbit;       // [dim]
    std::vector<int64_t> col_off;         // [dim+1] offset into coef (length = orbit size)
    std::vector<cplx> coef;               // concatenated column vectors on their orbit
    std::vector<int64_t> star_col;        // [n_stars+1] column range of each star
};
int build_basis(const Tables& t, int mu, Basis& out);
int build_basis_weighted(const Tables& t, const std::vector<double>& w, Basis& out);
int partner_matrices(const Tables& t, int mu, int& d, std::vector<double>& gam);
// outs[i] = (sum_s ws[i][s] Gamma~(s)) u for every i, in one pass over the orbits
int transfer_bases(const Tables& t, const Basis& u, const std::vector<std::vector<double>>& ws,
                   const std::vector<Basis*>& outs);

// ---------------------------------------------------------------------------
// device-side view of the system (passed by value to kernels)
// ---------------------------------------------------------------------------
struct DevSys {
    const double2* coef;   // [nk][nb][npw_max]
    const double* eps;     // [nk][nb]
    const double2* w;      // [nk][ng_max][ng_max]
    const int* gk;         // [nk][npw_max][3]
    const int* gq;         // [nk][ng_max][3]
    const int* npw;        // [nk]
    const int* ng;         // [nk]
    const int* kidx;       // [nk][3]
    const short* box;      // [nk][bvol] index of m in S_k or -1
    int blo[3], bdim[3];
    int64_t bvol;
    int n1, n2, n3, nk, nv, nc, nb, npw_max, ng_max;
    int g0;                // index of G = 0 in the sphere of q = 0
    double inv_vol;        // 1 / (Nk V_uc)
    double recip[9];       // row-major reciprocal basis (columns b_j)
    double qhat[3];
    double v_uc, scissor;
};

// one k pair of the direct term and where its B x B block goes
struct PairTask {
    int32_t k, kp;
    int32_t row0, col0;     // block origin inside the tile
    int64_t xoff;           // tile origin in the arena (elements)
    int32_t ld;             // tile leading dimension (column-major)
    int32_t flags;          // bit 0: also write the mirrored (conjugate) block; bits 1..: instance index
};

// one system of a direct-kernel launch (several in a batched launch)
struct __align__(16) DirectInst {
    DevSys S;
    const void* coef;       // coefficients in the launch precision (FP64 or FP32 complex)
    const void* w;          // W(q) in the launch precision
};

// a group of k pairs with the same q = k - k' (tensor-core direct term)
struct TcGroup {
    int32_t first, count, q;   // range in the q-sorted task list
    int32_t inst;              // system of the launch (index into its TcInst array)
};

// one system of a tensor-core launch
struct __align__(16) TcInst {
    DevSys S;
    const float2* coef;     // FP32 coefficients
    const void* wemb;       // W(q) embeddings (bf16 or fp16 hi and lo planes)
    const int* wexp;        // their per-q scale exponents
    int32_t ngp, kg;        // NG padded to 16; pairs per group
    int32_t pad[2];
};

// a star-pair tile for the projection kernels
struct TileTask {
    int64_t xoff, yoff;     // tile origins (elements) of X and Y
    int32_t rows;           // |a| * B  (leading dimension of X and Y)
    int32_t cols;           // |b| * B
    int32_t star_a, star_b;
    int64_t ca0, ca1;       // H_mu column range of star a
    int64_t cb0, cb1;       // H_mu column range of star b
};

// device copy of one irrep basis
struct DevBasis {
    int64_t dim;
    const int* col_orbit;       // [dim]
    const int64_t* col_off;     // [dim+1]
    const double2* coef;        // concatenated
    const float4* coef_df;      // the same in double-float (real hi, lo, imaginary hi, lo)
    const int64_t* orbit_off;   // [n_orbits+1]
    const int64_t* members;     // product indices
    const int* member_loc;      // local row of each member inside its star tile
};

// kernel launchers (kernels.cu); all on the given stream
int launch_rotmap(const DevSys& s, const int* rk, const double* tau, const int* rotk, int nops,
                  int* perm, double2* phase, cudaStream_t st);
int launch_gamma(const DevSys& s, int nops, const int* rotk, const int* perm, const double2* phase,
                 const int* ent, int64_t n_ent, double2* out, cudaStream_t st);
int launch_pairdens(const DevSys& s, const int* k, const int* kp, int64_t npairs, int bands,
                    int exchange_layout, double2* out, cudaStream_t st);
// the same in FP32 from the FP32 copy of the coefficients (pair layout only)
int launch_pairdens32(const DevSys& s, const float2* coef32, const int* k, const int* kp, int64_t npairs, int bands,
                      float2* out, cudaStream_t st);
// direct term (direct.cu): prec32 = 0 -> FP64 (coef/w double2, X double2), 1 -> FP32 (float2).
// One system, passed as a kernel parameter:
int launch_direct(const DirectInst& one, int prec32, const PairTask* tasks, int64_t ntasks, void* X, cudaStream_t st);
// Persistent form for batches: one launch of sms x (CTAs per SM, capped by ctas_per_sm when > 0)
// CTAs taking the tasks of all systems from a work queue (counter: device, zero before the launch);
// insts (device) holds the systems, task.flags >> 1 indexes them; smax: any system's (nb, nv, nc,
// npw_max, ng_max) maxima, for the shared-memory size; threads 128 or 256
int launch_direct_persistent(const DirectInst* insts, const DevSys& smax, int prec32, const PairTask* tasks,
                             int64_t ntasks, unsigned long long* counter, int threads, int ctas_per_sm, void* X,
                             cudaStream_t st);

// rotated direct-term blocks (rotate.cu, Eq. Wtrafo)
struct RotSys {
    const void* gam;        // Gamma(s) multiplet blocks [nops][gps] in the launch precision
    const int64_t* koff;    // [nk+1] offset of k's blocks within one operation
    const int64_t* boff;    // [nk*nb] offset of a band's multiplet block from koff[k]
    const int* mfirst;      // [nk*nb] first band of the band's multiplet at k
    const int* msize;       // [nk*nb] size of that multiplet
    int64_t gps;            // entries per operation
    int nk, nb, nv, nc;
};
struct RotTask {
    int64_t src;            // seed block origin in the arena (elements)
    int64_t dst;            // target block origin
    int64_t dstm;           // origin of its mirror (conjugate transpose), if flags & 1
    int32_t k, kp;          // target pair
    int32_t s;              // operation with s k = seed k, s k' = seed k'
    int32_t ld;             // tile leading dimension
    int32_t flags;          // bit 0: write the mirror; bits 1..: instance index
    int32_t pad;
};
int launch_rotate(const RotSys& one, int prec32, const RotTask* tasks, int64_t n, void* X, cudaStream_t st);

// A star-pair tile whose rotated k pairs the device enumerates (Eq. Wtrafo):
// its pairs (i, j) (members i of star a, j of star b; j >= i when a == b)
// are numbered row by row from pair_off; the seeds are the pairs (0, j) with
// j its own little-orbit representative, every other pair is written as a
// RotTask at rot_off + (its number in the tile - the seeds before it).
struct RotTile {
    int64_t xoff;       // tile origin in the arena (elements)
    int64_t pair_off;   // number of the tile's first pair in the batch
    int64_t rot_off;    // index of its first rotated pair in the RotTask list
    int32_t rows;       // tile rows (= leading dimension) = |star a| x B
    int32_t a, b;       // stars
    int32_t tri;        // a == b
    int32_t seeds;      // seeds of the tile
    int32_t rep_off;    // offset of the tile's per-member arrays of star b
};
// device copies of the group and star tables the enumeration reads
struct RotTables {
    const int* rotk;          // [nops][nk] index of s k
    const int* mult;          // [nops][nops] index of s1 s2
    const int* inv;           // [nops]
    const int* s_k;           // [nk] operation taking the representative of k's star to k
    const int* pos_in_star;   // [nk]
    const int* star_k;        // members of all stars, star by star
    const int* star_off;      // [nstars + 1]
    int nops, nk, B;
};
// jr[rep_off + j]: position in star b of the little-orbit representative of
// member j; gop[rep_off + j]: the little-group operation taking j to it;
// seedpre[rep_off + j]: seeds (0, j') with j' < j.  An inconsistent table
// sets bit 1 of *status (the tile's tasks are then incomplete).
int launch_rot_tasks(const RotTables& g, const RotTile* tiles, int ntiles, int64_t npairs, const int* jr,
                     const int* gop, const int* seedpre, RotTask* out, int* status, cudaStream_t st);
int launch_rotate_multi(const RotSys* systems, int bmax, int prec32, const RotTask* tasks, int64_t n, void* X,
                        cudaStream_t st);
// dynamic shared memory of the direct kernel for a system
size_t direct_smem(const DevSys& s, int prec32);
int launch_narrow(const double2* in, float2* out, int64_t n, cudaStream_t st);
// complex double-float copy (real hi, lo, imaginary hi, lo) of n complex doubles
int launch_to_df(const double2* in, float4* out, int64_t n, cudaStream_t st);
// x32: FP32 tiles (double-float products); ydf: write Y in double-float (float4) for
// launch_project_left with ydf
int launch_project_right(const DevBasis& b, const TileTask* tiles, int ntiles, int x32, const void* X,
                         double2* Y, int64_t max_rows, int64_t max_cols, cudaStream_t st, int ydf = 0);
// de: eps_c - eps_v per product index (or null to skip the diagonal); w_div:
// device pointer to W^div, subtracted on the diagonal with it
int launch_project_left(const DevBasis& b, const TileTask* tiles, int ntiles, const double2* Y,
                        const double2* Pmu, const double* vbar, int ng0, double xscale, const double* de,
                        const double* w_div, double2* H, int64_t ld, int64_t max_ca, int64_t max_cb, cudaStream_t st,
                        int ydf = 0, const float4* Pt = nullptr);
// Pt[i][g] = sqrt(vbar[g]) Pmu[i][g] in double-float, for launch_project_left with ydf
int launch_exchange_df(const double2* Pmu, const double* vbar, int64_t n, int ng0, float4* out, cudaStream_t st);
int launch_diag_full(const double* de, int64_t N, const double* w_div, double2* H, int64_t ld, cudaStream_t st);
// w = a - b * (*sum), on the stream
int launch_wdiv_finalize(const double* sum, double a, double b, double* w, cudaStream_t st);
void note_launch();
// split-precision tensor-core direct term (direct_tc.cu)
// split-precision support for a system: NG padded to 16 (ngp), the shared memory of a CTA and the
// number of k pairs per group (kg, at most 4); EUNSUPPORTED when the sizes do not fit
int tc_supported(const DevSys& s, int& ngp, size_t& smem, int* kg = nullptr);
// split-precision W(q) embeddings (fp16 != 0: fp16 hi + lo, else bf16) and their per-q scale exponents
int launch_wemb(const DevSys& s, int ngp, int fp16, void* out, int* wexp, cudaStream_t st);
// dynamic shared memory of a system's plan with kg pairs per group (0 if it does not fit)
size_t tc_smem(const DevSys& s, int ngp, int kg);
// one persistent launch over groups of one or more systems (insts: device; group.inst indexes it);
// smem: the largest plan of the systems; counter: device, zero before the launch;
// wait_polls: polls of an mbarrier wait before it gives up (negative: the default)
int launch_direct_tc(const TcInst* insts, int fp16, size_t smem, const PairTask* tasks, const TcGroup* groups,
                     int64_t ngroups, unsigned long long* counter, void* X, int* status, cudaStream_t st,
                     long wait_polls = -1);
int launch_exchange_project(const DevBasis& b, const double2* P, int ng0, double2* Pmu, cudaStream_t st);
int launch_exchange_full(const double2* P, const double* vbar, int ng0, int64_t N, double xscale,
                         double2* H, int64_t ld, cudaStream_t st);
int launch_basis_dense(const DevBasis& b, double2* U, int64_t ld, cudaStream_t st);
int launch_dipoles(const DevSys& s, double2* B, cudaStream_t st);
int launch_bmu(const DevBasis& b, const double2* B, double2* Bmu, cudaStream_t st);
int launch_oscillators(const double2* a, int64_t lda, int64_t dim, const double2* Bmu, int nparts, double* osc,
                       cudaStream_t st);
// tridiag.cu: levels and strengths through a tridiagonal reduction from the dipole direction
size_t tridiag_scratch_bytes(int64_t n);
int tridiag_max_dim();
int launch_gram(const double2* b, int64_t n, int np, double2* G, cudaStream_t st);
// ev0 / ev1 (may be null) are recorded around the reduction kernel
// wait_polls: polls of a grid barrier before it gives up (negative: the default)
int launch_tridiag_spectrum(double2* h, int64_t n, const double2* b, double scale, void* scratch, double* omega_out,
                            double* osc, double* wsum, int* err, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1,
                            long wait_polls = -1, int variant = 0, int* used = nullptr);
// variant: 0 the reduction with the block in shared memory when it fits, else the blocked
// (panel) reduction with the columns in global memory and its panel-end update on the tensor
// cores; 1 the blocked reduction always (tensor-core update); 2 the blocked reduction always,
// with the panel-end update on the CUDA cores (double-float) inside its single launch.
// *used (optional): 0 the shared-memory reduction ran, 1 the blocked one with the tensor-core
// update, 2 the blocked one with the CUDA-core update
// her2k_tc.cu: the panel-end update A -= V W^H + W V^H (rows and columns >= k0 of the n x n
// double-float block; V, W [32][n]) from exact bf16 digit GEMMs on the tensor cores; columns
// below resident_from are read and written with evict-first hints; status is raised when a
// bounded wait gives up
size_t panel_update_tc_bytes(int64_t n);
// tridiag2.cu: the two-stage reduction (start reflector, dense -> band 32 by panels with the
// tensor-core rank-64 update, band -> tridiagonal by bulge chasing) of the FP64 block A (n x n,
// rewritten in double-float in place) to d, e; V, W [32][n] and tc_scratch as for the panel
// update, scratch of tridiag2_bytes(n)
size_t tridiag2_bytes(int64_t n);
// zgemm_tc.cu: Z = A22 V (rows and columns r1.. of the n x n double-float block, V [32][n]) from
// exact bf16 digit GEMMs on the tensor cores, K split nsplit ways into zpart[nsplit][m][32]
size_t zgemm_tc_bytes(int64_t n);
int zgemm_tc_splits(int64_t m, int sms);
int launch_zgemm_tc(const float4* A, int64_t n, int r1, int m, const float4* V, void* scratch, float4* zpart,
                    int nsplit, int* status, cudaStream_t st, long wait_polls);
int launch_tridiag2(float4* A, int64_t n, const double2* v0, const double* beta0, double* d, double* e, float4* V,
                    float4* W, void* tc_scratch, void* scratch, int* err, cudaStream_t st, long wait_polls);
int launch_panel_update_tc(float4* A, int64_t n, int k0, int resident_from, const float4* V, const float4* W,
                           void* scratch, int* status, cudaStream_t st, long wait_polls);
// lanczos.cu: the Lanczos recurrence on a Hermitian block from conj(b) (Lanczos-Haydock, Sec. IV)
size_t lanczos_scratch_bytes(int64_t n, int m);
int lanczos_max_dim();
// steps: requested; on return *done (host) = steps performed, alpha [done], beta [done] (beta[j] couples j-1, j)
// wait_polls: polls of a grid barrier before it gives up (negative: the default)
int launch_lanczos(const double2* h, int64_t ld, int64_t n, const double2* b, int steps, void* scratch,
                   double** alpha, double** beta, int* done, cudaStream_t st, long wait_polls = -1);
// T_m dense (k x k column-major) from alpha and beta1 (beta1[j] couples j, j + 1); Gauss weights
// scale V[0][j]^2 from its eigenvector matrix V
int launch_tm_dense(const double* alpha, const double* beta1, int k, double* T, cudaStream_t st);
int launch_tm_weights(const double* V, int k, double scale, double* w, cudaStream_t st);
// Im eps from the continued fraction of (alpha, beta1) with weight norm2 and prefactor pref
int launch_cf_spectrum(const double* alpha, const double* beta1, int k, double norm2, const double* omega,
                       int64_t n_omega, double eta, double pref, double* im, cudaStream_t st);
// loss.cu: longitudinal levels (Eq. secular) and strengths (Eq. eigenvec_xi)
size_t loss_scratch_bytes(int64_t n);
int launch_loss_levels(const double* Om, const double* osc, int64_t n, double alpha, void* scratch, double* out_l,
                       double* out_w, cudaStream_t st);
int launch_spectrum(const double* Om, const double* osc, int64_t dim, const double* omega,
                    int64_t n_omega, double eta, double pref, double* im, cudaStream_t st);
// recip_and_lattice: reciprocal basis then lattice, both row-major 3x3.  With
// nops > 0, Mx [nops][9] is the point group acting on the integer coordinates
// of Q = sum X_j b_j / n_j (row-major) and the sum runs over one point per
// orbit (the caller has checked that L is invariant); nops = 0: every point.
// scratch of the orbit sum: the per-column arrays (wdiv_sym_bytes).  Nothing
// of the sum returns to the host: out receives it on the stream.
struct WdivScratch {
    void* base = nullptr;   // wdiv_sym_bytes() of device memory
};
size_t wdiv_sym_bytes(const double* lattice, const int* n, double qmax, double delta);
int launch_wdiv(const double* recip_and_lattice, const int* n, const double* L, double b, double qmax,
                double delta, double* partial, int64_t npartial_max, double* out, cudaStream_t st, int nops = 0,
                const int* Mx = nullptr, WdivScratch* sym_scratch = nullptr);
int64_t wdiv_partials(const double* lattice, const int* n, double qmax, double delta);
// points of one lattice column of that sum (the loop length of one thread)
int64_t wdiv_column_length(const double* lattice, const int* n, double qmax, double delta);
int launch_count_overlap(const DevSys& s, const PairTask* tasks, int64_t ntasks, unsigned long long* out,
                         cudaStream_t st);
int64_t launches_total();

}  // namespace bse
