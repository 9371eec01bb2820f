/*
 * bse.h - C ABI of the GB300 symmetry-reduced Bethe-Salpeter block builder.
 *
 * Computes, on one GPU, the symmetry-adapted block of the electron-hole
 * Hamiltonian of Stöhler, Blügel and Friedrich, "Efficient all-electron
 * Bethe-Salpeter implementation using crystal symmetries":
 *
 *   H = diag(eps_ck - eps_vk) + spin * K^x - K^d            (Eq. BSE-eigval)
 *   H_mu = U_mu^dagger H U_mu                               (Eqs. projection,
 *                                                            transformationU)
 *
 * in a plane-wave basis, and the optical spectrum of one block
 * (Eqs. macro_diel, reducible_polar, oscillatorA, oscillator).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Atomic units (bohr, hartree).  Complex numbers are interleaved
 *    (re, im) doubles.  Matrices are row-major unless stated otherwise.
 *  - Lattice L: 3x3, row-major, columns are a1, a2, a3.  A symmetry
 *    operation {R|t} maps fractional positions x -> R x + t (Eq. sk, sphi
 *    with alpha = 0); it maps reciprocal fractional vectors y -> R^{-T} y.
 *  - Gamma-centred mesh n1 x n2 x n3: f_k = (i/n1, j/n2, l/n3),
 *    k = (i*n2 + j)*n3 + l.  The same mesh indexes q = k - k'.
 *  - A plane wave of band coefficient c_kn(p) has the full wave vector
 *    p = f_k + m (m integer, reciprocal fractional coordinates).
 *  - Bands 0..nv-1 are occupied (v), nv..nv+nc-1 unoccupied (c).
 *    Product index I = (k*nv + v)*nc + c  (Eq. 2p-product-basis).
 *  - Irreps are numbered in the canonical order returned by bse_tables:
 *    ascending (dimension, then character vector over operations).
 *  - All device work runs on the CUDA stream given to bse_create, in stream
 *    order; functions return once the work is enqueued unless stated.
 *  - Every function returns BSE_OK (0) or a negative status; the message of
 *    the last failure of the calling thread is bse_last_error().
 */
#ifndef BSE_GB300_H
#define BSE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bse_ctx bse_ctx;   /* opaque, library-owned; not thread-safe */
typedef struct bse_batch bse_batch;   /* opaque: a batched build of several contexts */

enum {
    BSE_OK = 0,
    BSE_EINVAL = -1,       /* invalid argument (sizes, pointers, indices) */
    BSE_ENOMEM = -2,       /* device or host allocation failed */
    BSE_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    BSE_ESYMM = -4,        /* inputs break the symmetry (non-unitary band rotation,
                              inconsistent orbits, block dims not summing to N) */
    BSE_ETIMEOUT = -5,     /* a bounded device wait gave up */
    BSE_EUNSUPPORTED = -6, /* a case outside what is implemented */
    BSE_ESOLVER = -7       /* the dense eigensolver failed */
};

/* precision of the direct term: FP64 throughout; FP32 CUDA-core arithmetic;
   or BF16_SPLIT / FP16_SPLIT: pair densities in FP32 on CUDA cores and both
   dense contractions (W(q) conj(rho_vv') and rho_cc'^T T) on the tensor cores
   with every operand split into a 16-bit hi + lo pair (bf16: 2 x 8
   significant bits; fp16: 2 x 11 bits, each operand scaled by an exact power
   of two into fp16's range) and three products accumulated in FP32.  The
   diagonal and W^div stay FP64; the projection and the exchange are FP64
   in the FP64 build and, for the FP32 tiles of the other modes, formed in
   double-float (a pair of floats, 48-bit significand: products exact, sums
   far below the tiles' own error). */
enum { BSE_FP64 = 0, BSE_BF16_SPLIT = 1, BSE_FP16_SPLIT = 2, BSE_FP32 = 3 };

/* terms of H to include (bit mask) */
enum { BSE_TERM_DIAG = 1, BSE_TERM_EXCHANGE = 2, BSE_TERM_DIRECT = 4, BSE_TERM_ALL = 7 };

/* band sets of bse_pairdens */
enum { BSE_BANDS_CC = 0, BSE_BANDS_VV = 1, BSE_BANDS_CV = 2 };

/*
 * bse_system: one crystal, its symmetry, its band coefficients and W(q).
 * Everything is copied at bse_create; the caller keeps ownership.
 * Pointers marked [loc] are device pointers when device_inputs != 0, host
 * pointers otherwise; all other pointers are host pointers.
 */
typedef struct {
    double lattice[9];       /* L, row-major, columns a1 a2 a3 (bohr) */
    int32_t n_ops;           /* number of space-group operations modulo lattice translations */
    const int32_t* rot;      /* [n_ops][3][3] R (row-major) in lattice coordinates */
    const double* tau;       /* [n_ops][3] fractional translation t */
    int32_t mesh[3];         /* n1, n2, n3 */
    int32_t nv, nc;          /* occupied / unoccupied bands per k */
    int32_t npw_max;         /* capacity of the plane-wave axis of coef and gk */
    const int32_t* npw;      /* [Nk] plane waves at k */
    const int32_t* gk;       /* [Nk][npw_max][3] integer m of p = f_k + m; any order */
    const double* coef;      /* [loc] [Nk][nv+nc][npw_max] complex c_kn(p), orthonormal bands */
    const double* eps;       /* [loc] [Nk][nv+nc] band energies (Ha) entering H */
    int32_t ng_max;          /* capacity of the G axis of W and gq */
    const int32_t* ng;       /* [Nk] number of Q = f_q + G at q */
    const int32_t* gq;       /* [Nk][ng_max][3] integer G of Q = f_q + G; sphere must contain G = 0 at q = 0 */
    const double* w;         /* [loc] [Nk][ng_max][ng_max] complex W_{QQ'}(q), row Q, column Q'.
                                At q = 0 the head and wings are ignored (Sec. III.B). */
    double eps_inf[9];       /* dielectric tensor L of Eq. Wdiv, row-major */
    double w_div;            /* head correction W^div (Ha); NaN: computed (Eqs. Wdiv,
                                divergence_int, divergence_sum, b = 0.005) */
    double qhat[3];          /* light polarisation (Cartesian, unit vector) */
    double scissor;          /* eps0_c = eps_c - scissor in Eq. oscillator */
    int32_t spin_factor;     /* 2 for a non-magnetic system without SOC */
    int32_t device_inputs;   /* 0: [loc] pointers are host pointers; 1: device pointers */
} bse_system;

/*
 * bse_create - validate the system, build the symmetry tables (stars,
 * little groups, characters, orbits; Sec. III.C), the band rotations
 * Gamma(s) (Eq. Ts) and the canonical orthonormal basis of every irrep
 * (Eq. projection followed by two-pass modified Gram-Schmidt per orbit; the
 * paper uses an SVD, whose basis is not unique), and compute W^div if
 * requested.  stream: a cudaStream_t, or NULL for the default stream.
 * On success *out owns device memory until bse_destroy.  Blocks until the
 * set-up work has finished.  Device memory of contexts comes from the
 * device's stream-ordered memory pool (cudaMallocAsync on the context's
 * stream); bse_create raises that pool's release threshold to 64 GiB, so
 * memory freed by one context is reused by the next without a driver
 * allocation.  The builds' tile arenas take up to a sixth of the free device
 * memory (at most 32 GiB each; environment variable BSE_ARENA_MB fixes the
 * budget), so that a workload's tiles fit one batch when there is room.
 * Errors: EINVAL (sizes, non-unimodular R, mesh not invariant, G = 0 missing),
 * ESYMM (operations not a group, sphere not closed under an operation,
 * non-unitary Gamma, block dimensions not summing to N), EUNSUPPORTED
 * (complex characters), ENOMEM, ECUDA.
 */
int bse_create(bse_ctx** out, const bse_system* sys, void* stream);

/* bse_destroy - wait for the context's stream, then free everything owned
 * by ctx (device memory returns to the device's memory pool; NULL is
 * allowed). */
int bse_destroy(bse_ctx* ctx);

/* Message of the last failure on the calling thread ("" if none). */
const char* bse_last_error(void);

/*
 * bse_tables_view: read-only host views into tables owned by ctx (valid
 * until bse_destroy).  These are integer-exact and match the oracle's.
 */
typedef struct {
    int32_t n_ops, nk, n_stars, n_irreps, n_orbits;
    int64_t n_product;            /* N = Nk * nv * nc */
    const int32_t* rotk;          /* [n_ops][nk] mesh index of s k */
    const int32_t* star_of_k;     /* [nk] star of k; stars numbered by their lowest k */
    const int32_t* star_rep;      /* [n_stars] lowest k of the star */
    const int32_t* s_k;           /* [nk] lowest operation index s with s star_rep = k */
    const int32_t* class_of_op;   /* [n_ops] conjugacy class (numbered by lowest op) */
    const int32_t* chi;           /* [n_irreps][n_ops] characters (Eq. LOT holds) */
    const int32_t* irrep_dim;     /* [n_irreps] d_mu */
    const int32_t* bright;        /* [n_irreps] multiplicity in the polar-vector representation */
    const int64_t* block_dim;     /* [n_irreps] dimension of H_mu */
    const int32_t* orbit_of;      /* [N] orbit of each product index; orbits ordered by lowest member */
    double w_div;                 /* head correction used on the diagonal (Ha) */
    const int64_t* partner_dim;   /* [n_irreps] dim_mu / d_mu where a partner block exists, else 0 */
    const int32_t* fold;          /* [n_ops][nk][3] integer G-bar with R^{-T} f_k = f_{sk} + G-bar (Eq. sk) */
    int32_t npw_max, ng_max;      /* capacities of the sphere arrays below */
    const int32_t* npw;           /* [nk] |S_k|: plane waves of the coset sphere of k */
    const int32_t* gk;            /* [nk][npw_max][3] integer m of p = f_k + m in S_k, in the order of bse_system */
    const int32_t* ng;            /* [nk] |S_q|: points Q = f_q + G of the sphere of W(q) */
    const int32_t* gq;            /* [nk][ng_max][3] integer G of S_q, in the order of bse_system */
} bse_tables_view;

/*
 * bse_tables - the symmetry tables the construction works from (Sec. III.C):
 * the rotated mesh points s k and their folds (Eq. sk), the stars with their
 * representatives and the operations s_k reaching each member, the
 * conjugacy classes and characters (computed, Burnside-Dixon; Eq. LOT
 * holds), the irreps' multiplicities in the polar-vector representation
 * (Sec. III.D: the optically active irreps), the block dimensions
 * dim_mu = Tr P_mu (Eq. projection: d_mu/|S| sum_s chi_mu(s)^* Tr Gamma~(s)),
 * the orbits of the product basis, the coset spheres S_k and S_q, W^div, and
 * the partner dimensions.  The first call also forms the irrep matrices of
 * every irrep that has them (for the partner dimensions); it returns ESYMM
 * when their row projector's trace Tr P_11 is not dim_mu / d_mu (inputs that
 * break the symmetry in a way bse_create's checks do not see), EINVAL for a
 * null argument.  Views stay valid until bse_destroy.
 */
int bse_tables(const bse_ctx* ctx, bse_tables_view* out);

/*
 * bse_pairdens - pair densities (Eq. w_interaction in plane waves)
 *   rho_nn'(k, k'; Q) = sum_{p' in S_k'} conj(c_kn(p' + Q)) c_k'n'(p'),
 *   Q = f_q + G over the sphere of q = k - k'.
 * bands: BSE_BANDS_CC (n, n' conduction), BSE_BANDS_VV, or BSE_BANDS_CV
 * (n conduction, n' valence; with k = k' these are the exchange vectors
 * m^k_cv(G) of Eq. v_scalar).
 * prec: BSE_FP64 (FP64 arithmetic, out complex128) or the precision of a
 * mixed build, BSE_FP32, BSE_BF16_SPLIT or BSE_FP16_SPLIT: the densities
 * those builds use, FP32 arithmetic on the FP32 copy of the coefficients
 * (out complex64; the split modes split them into 16-bit pairs only inside
 * the tensor-core kernel).
 * k, kp: host arrays [npairs]; out_dev: device [npairs][n][n'][ng_max]
 * of that type, entries with G index >= ng(q) set to zero; caller-owned.
 * Errors: EINVAL (bands, prec, a k index out of range, null pointers).
 */
int bse_pairdens(bse_ctx* ctx, const int32_t* k, const int32_t* kp, int64_t npairs,
                 int32_t bands, int32_t prec, void* out_dev);

/*
 * bse_build_block - H_mu = U_mu^dagger H U_mu for irrep mu, never forming
 * the full H: direct-term tiles of each pair of k stars are projected at
 * once (Sec. III.C.5), the exchange term is applied in the projected form
 * (U_mu^dagger P) vbar (U_mu^dagger P)^dagger (Eq. v_scalar), the diagonal
 * eps_c - eps_v - W^div in FP64.  terms: BSE_TERM_* mask.
 * prec: BSE_FP64, BSE_FP32, BSE_BF16_SPLIT or BSE_FP16_SPLIT (see the
 * precision enum); the split modes need NG_max <= 128, nv <= 8, nc <= 8 and
 * their operands within 227 KB of shared memory per CTA, and return
 * EUNSUPPORTED otherwise.  ETIMEOUT if a
 * bounded wait of the tensor-core kernel gave up (the context stays usable).
 * h_dev: device, complex128, column-major dim x dim with leading dimension
 * ld >= dim; the full Hermitian matrix is written.  irrep = BSE_IRREP_ALL
 * writes the blocks of all irreps from one direct pass (as bse_build_blocks),
 * packed one after another in irrep order: block mu is dim_mu x dim_mu,
 * column-major with leading dimension dim_mu, at element offset
 * sum_{nu < mu} dim_nu^2 (ld is ignored).  Scratch is library-owned.
 */
enum { BSE_IRREP_ALL = -1 };

/* bse_block_dim - dim_mu = Tr P_mu of an irrep (N for BSE_IRREP_ALL): the
 * trace of the projector of Eq. projection, d_mu/|S| sum_s chi_mu(s)^*
 * Tr Gamma~(s), from the band rotations of the k points each operation fixes
 * (Sec. III.C.4); integer-exact.  Errors: EINVAL (irrep out of range). */
int bse_block_dim(const bse_ctx* ctx, int32_t irrep, int64_t* dim);

int bse_build_block(bse_ctx* ctx, int32_t irrep, int32_t prec, uint32_t terms,
                    void* h_dev, int64_t ld);

/*
 * bse_build_partner_block - the block of the first partner of an irrep,
 * H_mu^(1) = U_1^dagger H U_1, where U_1 spans the range of the row projector
 *   P_11 = d_mu/|S| sum_s Gamma_mu(s)_11 Gamma~(s)
 * with real orthogonal irrep matrices Gamma_mu(s): for an irrep contained
 * once in the polar-vector representation (the optically active ones: T1u
 * of Oh, E1u and A2u of D6h) the Cartesian rotations restricted to its
 * Cartesian subspace; for a one-dimensional irrep its character; for any
 * other irrep a canonical copy inside the left regular representation (the
 * lowest eigenspace of a fixed generic element of its commutant, its basis
 * fixed by Gram-Schmidt over the projected unit vectors).  Sec. III.C.3 (the
 * blocks H^{mu i}_{mu j} are multiples of the identity) makes H_mu unitarily
 * equivalent to d_mu copies of H_mu^(1): its eigenvalues are those of H_mu,
 * each once instead of d_mu times, and the eigensolver works on a matrix
 * d_mu times smaller.  Dimension partner_dim[irrep] of bse_tables; arguments
 * as bse_build_block.  Errors: ESYMM if the irrep matrices cannot be formed
 * (partner_dim is 0 then).
 */
int bse_build_partner_block(bse_ctx* ctx, int32_t irrep, int32_t prec, uint32_t terms,
                            void* h_dev, int64_t ld);

/*
 * bse_build_blocks - several blocks in one build: target i is the block of
 * irrep[i] (partner == NULL or partner[i] == 0) or its partner block
 * (partner[i] != 0), written to h_dev[i] (device, complex128 column-major,
 * leading dimension ld[i]; may be NULL when the block is empty).  Sec. III.C
 * decomposes H into the blocks of all irreps; their direct terms share the
 * same k-pair matrix elements, so the direct kernel runs once per star pair
 * and every target projects the same tiles (Eqs. transformationU, Hblock).
 * irrep, partner, h_dev and ld are host arrays of n entries, borrowed for the
 * call.  The result of each target equals that of bse_build_block or
 * bse_build_partner_block with the same arguments.  Errors as
 * bse_build_block, reported for the first target that fails.
 */
int bse_build_blocks(bse_ctx* ctx, int32_t n, const int32_t* irrep, const int32_t* partner, int32_t prec,
                     uint32_t terms, void* const* h_dev, const int64_t* ld);

/*
 * Batched builds (no counterpart in the paper, which treats one crystal at a
 * time): one block for each of n independent contexts on the same device
 * and stream.  The direct terms of all contexts run in one launch of a
 * persistent kernel (a grid sized to the GPU taking the k-pair tasks of all
 * contexts, or for the split modes their groups of k pairs sharing one q,
 * from a device work queue, longest first; every task carries the index of
 * its context's system); the exchange and projections follow per context.
 * An autotuner times the candidate tile shapes on the batch's own tasks at
 * bse_batch_create (pairs per CTA per class of instances for the split modes,
 * threads per CTA otherwise; the choices of a class are kept for the
 * process).  The sequence is captured once into a CUDA graph, so a build of
 * the whole batch is one graph launch.
 *
 * bse_batch_create - plan the batch: target i is the block of irrep[i] of
 *   ctxs[i] (partner == NULL or partner[i] == 0) or its partner block
 *   (partner[i] != 0), written to h_dev[i] with leading dimension ld[i];
 *   prec any of the precision enum.  All arrays are host arrays of n entries,
 *   borrowed for the call; the contexts and the output buffers must outlive
 *   the batch.  Builds the bases, uploads the plan, allocates one X arena
 *   for all contexts (the sum of their direct-term tiles) and captures the
 *   graph; blocks until done.  Errors: as bse_build_blocks; EINVAL if the
 *   contexts do not share one stream; EUNSUPPORTED where a split mode does
 *   not support an instance's sizes.
 * bse_batch_run - launch the graph on the contexts' stream (asynchronous).
 *   The result of target i equals that of bse_build_blocks on ctxs[i] alone.
 * bse_batch_kernels - number of kernel launches one run performs.
 * bse_batch_tuning - the autotuner's choices for the batch, as a JSON object
 *   (NUL-terminated, truncated to len - 1 characters): for the split modes the
 *   k pairs per CTA of each class of instances (same nv, nc, NG and sphere
 *   capacities) with the measured time of each candidate, for FP32 / FP64 the
 *   threads per CTA of the persistent direct kernel, and the X arena size.
 * bse_batch_destroy - wait for the stream and free the batch (NULL allowed);
 *   ETIMEOUT if a bounded wait of the tensor-core kernel gave up in any run.
 * bse_build_blocks_batched - create, run once, destroy.
 */
int bse_batch_create(bse_batch** out, bse_ctx* const* ctxs, int32_t n, const int32_t* irrep, const int32_t* partner,
                     int32_t prec, uint32_t terms, void* const* h_dev, const int64_t* ld);
int bse_batch_run(bse_batch* batch);
int bse_batch_kernels(const bse_batch* batch, int64_t* out);
int bse_batch_tuning(const bse_batch* batch, char* buf, int64_t len);
int bse_batch_destroy(bse_batch* batch);
int bse_build_blocks_batched(bse_ctx* const* ctxs, int32_t n, const int32_t* irrep, const int32_t* partner,
                             int32_t prec, uint32_t terms, void* const* h_dev, const int64_t* ld);

/*
 * bse_block_star_columns - column ranges of the k stars in the block of an
 * irrep (partner = 0) or in its partner block (partner = 1): the basis
 * vectors of star a are columns [out[a], out[a+1]); out is a host array of
 * n_stars + 1 entries.  Builds the basis if needed.
 */
int bse_block_star_columns(bse_ctx* ctx, int32_t irrep, int32_t partner, int64_t* out);

/*
 * bse_build_full - the unprojected H (N x N, complex128, column-major, ld
 * >= N, device) in FP64; meant for checks on small meshes.
 */
int bse_build_full(bse_ctx* ctx, uint32_t terms, void* h_dev, int64_t ld);

/*
 * bse_block_basis - the dense N x dim U_mu (complex128, column-major, ld >= N,
 * device), columns in block order.
 */
int bse_block_basis(bse_ctx* ctx, int32_t irrep, void* u_dev, int64_t ld);

/*
 * bse_dipoles - B_kvc = <phi_kv| -i qhat.grad |phi_kc> / (sqrt(V_uc)
 * (eps_c - scissor - eps_v)) (Eq. oscillator) for every product index;
 * b_dev: device [N] complex128.
 */
int bse_dipoles(bse_ctx* ctx, void* b_dev);

/*
 * bse_block_spectrum - eigensolution of H_mu (dense Hermitian FP64 solver,
 * or the eigenvector-free path of bse_set_solver) and the spectrum of the
 * block:
 *   B_lambda = a_lambda^T (U_mu^T B)                (Eq. oscillatorA)
 *   Im eps_M(w) = 4 pi spin / Nk sum_lambda |B_lambda|^2
 *                 [eta/((w - Omega)^2 + eta^2) - eta/((w + Omega)^2 + eta^2)]
 *                                                  (Eqs. macro_diel, reducible_polar)
 * h_dev: H_mu as written by bse_build_block (read only); omega_dev: device
 * [n_omega]; outputs (device, caller-owned): omega_out [dim] ascending
 * eigenvalues, osc [dim] |B_lambda|^2, im_eps [n_omega].
 * Errors: ESOLVER if the eigensolver reports failure.
 */
int bse_block_spectrum(bse_ctx* ctx, int32_t irrep, const void* h_dev, int64_t ld,
                       const double* omega_dev, int64_t n_omega, double eta,
                       double* omega_out, double* osc, double* im_eps);

/*
 * bse_partner_spectrum - as bse_block_spectrum for the partner block of
 * bse_build_partner_block: omega_out [partner_dim] are the distinct levels of
 * H_mu (each d_mu-fold in H_mu), osc [partner_dim] the oscillator strength of
 * each level summed over the d_mu partners, sum_i |a^T (U_i^T B)|^2 with
 * U_i = P_i1 U_1 (zero for an irrep outside the polar-vector
 * representation), and im_eps the spectrum of the whole block H_mu.
 */
int bse_partner_spectrum(bse_ctx* ctx, int32_t irrep, const void* h_dev, int64_t ld,
                         const double* omega_dev, int64_t n_omega, double eta,
                         double* omega_out, double* osc, double* im_eps);

/*
 * bse_block_spectrum_lanczos - the Lanczos-Haydock spectrum of a block
 * (Sec. IV: the spectrum without diagonalising, summed over the contributing
 * blocks), for blocks too large to reduce or when only Im eps is wanted.
 * steps of the Hermitian Lanczos recurrence on h_dev (the block of irrep, or
 * its partner block when partner != 0; device, complex128 column-major,
 * leading dimension ld, read only) from the dipole direction conj(U^T B),
 * without reorthogonalisation, build the tridiagonal T_m; im_eps is the
 * continued fraction of T_m (the Haydock spectrum), which reproduces the
 * first 2 m moments of the spectral measure; an invariant subspace ends the
 * recurrence early and the spectrum is then exact.  ritz_dev and weights_dev
 * are optional (both NULL or both device arrays of [steps]): the Ritz values
 * of T_m (ascending) and its Gauss weights sum_i |U_i^T B|^2 z_0(k)^2 (z_0
 * the first components of T_m's eigenvectors, from cuSOLVER's dense
 * symmetric eigensolver on the small T_m), zero beyond *steps_done, whose
 * Lorentzian sum equals im_eps.  *steps_done (host): the steps performed.  A
 * dark irrep (no dipole weight) gives an empty spectrum and *steps_done = 0.
 * Errors: EINVAL for steps outside [1, dim] or only one of ritz_dev and
 * weights_dev; EUNSUPPORTED for dim above 12 000 or non-parallel partner
 * projections; ETIMEOUT if a bounded grid barrier gave up; ESOLVER if the
 * dense eigensolver of T_m fails.
 */
int bse_block_spectrum_lanczos(bse_ctx* ctx, int32_t irrep, int32_t partner, const void* h_dev, int64_t ld,
                               int32_t steps, const double* omega_dev, int64_t n_omega, double eta,
                               double* ritz_dev, double* weights_dev, double* im_eps_dev, int32_t* steps_done);

/*
 * bse_set_solver - how bse_block_spectrum / bse_partner_spectrum obtain the
 * levels Omega_l and the oscillator strengths of Eqs. oscillator and
 * oscillatorA:
 *   BSE_SOLVER_DENSE   cuSOLVER zheevd (all eigenvectors), then |a_l^T b|^2.
 *   BSE_SOLVER_TRIDIAG a reflector maps c = conj(b) to a multiple of e_0,
 *                      a Householder reduction that keeps e_0 fixed turns
 *                      the block into a real tridiagonal T, and the strengths
 *                      are ||c||^2 times the squared first components of T's
 *                      eigenvectors (bisection for the levels, a twisted
 *                      factorisation per level for the components); no
 *                      eigenvector matrix is formed.  The reduction, the
 *                      bisection's refinement and the twisted pivots compute
 *                      in double-float (48-bit significand) on the FP32
 *                      pipe: levels within about n 2^-47 ||H_mu||, for
 *                      blocks whose entries lie below 2^50 in magnitude
 *                      (FP32's exponent range; Hartree-unit blocks are far
 *                      inside it).  Blocks of up to about 1200 rows are
 *                      reduced in shared memory (a column per CTA); larger
 *                      ones, up to n = 1800, with their columns in device
 *                      memory, by a blocked form of the same reduction
 *                      (panels of 32 reflectors: one pass of column dot
 *                      products per step; at the panel's end its rank-64
 *                      update of the trailing block on the tensor cores,
 *                      from an exact split of V and W into 8 bf16 digits,
 *                      digit-pair products summed in FP32 (exactly for the
 *                      leading groups), the groups combined in double-float);
 *                      from n = 1800 by the two-stage reduction of
 *                      BSE_SOLVER_TRIDIAG_TWOSTAGE.  Needs the partners'
 *                      projections b_i to be parallel (true for the partner
 *                      blocks of bse_partner_spectrum) and n <= 8192; the
 *                      sum of the weights must come out as 1 within 1e-8.
 *                      Otherwise the spectrum call fails (EUNSUPPORTED or
 *                      ESOLVER).  Exactly degenerate levels (the d_mu
 *                      copies in a whole block of a d_mu-dimensional irrep)
 *                      break the last condition.
 *   BSE_SOLVER_TRIDIAG_BLOCKED  as TRIDIAG with the blocked reduction at
 *                      every size (for checks and measurements).
 *   BSE_SOLVER_TRIDIAG_BLOCKED_DF  as TRIDIAG_BLOCKED with the panel-end
 *                      update on the CUDA cores in double-float (for checks
 *                      and measurements).
 *   BSE_SOLVER_TRIDIAG_TWOSTAGE  as TRIDIAG with a two-stage reduction at
 *                      every size: dense -> band of half-bandwidth 32 by
 *                      panels of 32 Householder reflectors (one pass of the
 *                      trailing block through a GEMM and the tensor-core
 *                      rank-64 update per panel), then band -> tridiagonal by
 *                      bulge chasing; every reflector keeps e_0 fixed.
 *   BSE_SOLVER_AUTO    (default) TRIDIAG for partner blocks, for blocks
 *                      of one-dimensional irreps and for blocks of irreps
 *                      outside the polar-vector representation (B_mu = 0
 *                      by symmetry: levels only, strengths 0), DENSE
 *                      otherwise and whenever a TRIDIAG condition fails.
 * bse_stats.solver reports the solver the last spectrum used.
 */
enum {
    BSE_SOLVER_AUTO = 0,
    BSE_SOLVER_DENSE = 1,
    BSE_SOLVER_TRIDIAG = 2,
    BSE_SOLVER_TRIDIAG_BLOCKED = 3,
    BSE_SOLVER_TRIDIAG_BLOCKED_DF = 4,
    BSE_SOLVER_TRIDIAG_TWOSTAGE = 5
};

/*
 * bse_set_seeds - direct term by seeds (on, the default) or pair by pair.
 * On: in each pair of k stars (a, b) the direct kernel computes only one k
 * pair per symmetry orbit, (k0, k'_r) with k0 the representative of star a
 * and k'_r the lowest k of each orbit of star b under the little group of
 * k0; every other pair (k, k') = (s^-1 k0, s^-1 k'_r) follows by Eq. Wtrafo,
 * K^d(k, k') = G(s,k)^dagger K^d(k0, k'_r) G(s,k'), with the two-particle
 * band rotations G of Eq. Ttilde (sums over degenerate multiplets only).
 * Off: every pair is computed.  Both give the same blocks to rounding.
 */
int bse_set_seeds(bse_ctx* ctx, int32_t on);
int bse_set_solver(bse_ctx* ctx, int32_t solver);

/*
 * bse_set_wait_limit - how long the context's kernels wait at a bounded
 * device wait (no counterpart in the paper: failure handling).  Every wait of
 * a device-wide step is bounded: the grid barriers of the tridiagonal
 * reduction and of the Lanczos recurrence, and the mbarrier waits of the
 * tensor-core direct kernel on its bulk copy and its MMAs.  A wait that gives
 * up raises an error flag, lets the copy or MMAs it waited for finish (the
 * default limit), frees its tensor memory and returns; the call then reports
 * ETIMEOUT and the context stays usable.  polls >= 0: a wait gives up after
 * that many polls (0: at once, which makes every such call report ETIMEOUT;
 * meant for tests of the failure path); polls < 0 (the default): seconds of
 * polling.  A batch (bse_batch_create) keeps the limits its contexts had when
 * it was created.
 */
int bse_set_wait_limit(bse_ctx* ctx, int64_t polls);

/*
 * bse_loss_spectrum - longitudinal excitons and the loss spectrum of a block
 * (Sec. III.D, "Excitonic energies and loss spectrum").  With the
 * unmodified Coulomb interaction H gains alpha B* B^T (Eq. epsinv_div),
 * alpha = 4 pi spin / N_k (B of Eq. oscillator carries 1/sqrt(V_uc)).  From
 * the levels Omega_l and strengths w_l = |B_l|^2 of bse_block_spectrum or
 * bse_partner_spectrum (omega_levels, osc: device, n entries, levels
 * ascending) the new levels are the roots of the secular equation
 * 1 - alpha sum_l w_l / (x - Omega_l) = 0 (Eq. secular): one in each gap
 * between consecutive levels with w_l > 1e-14 max w and one above the
 * highest; the other levels stay, with strength 0.  The strength of a
 * longitudinal exciton follows from its closed-form eigenvector
 * (Eq. eigenvec_xi): |B'_x|^2 = 1 / (alpha^2 sum_l w_l / (x - Omega_l)^2).
 * Outputs (device, caller-owned): omega_long [n] ascending, osc_long [n],
 * loss [n_omega] = -Im eps_M^-1(omega) = alpha sum_x |B'_x|^2
 * [eta/((omega-x)^2+eta^2) - eta/((omega+x)^2+eta^2)].  Asynchronous on the
 * context's stream.  Errors: EINVAL, EUNSUPPORTED (n > 2^20), ECUDA.
 */
int bse_loss_spectrum(bse_ctx* ctx, int64_t n, const double* omega_levels, const double* osc, const double* omega,
                      int64_t n_omega, double eta, double* omega_long, double* osc_long, double* loss);

/* Wait for all work on the context's stream; returns ECUDA on a device error. */
int bse_sync(bse_ctx* ctx);

/*
 * Measurement support (not part of the paper's method).
 *
 * bse_work: algorithmic work of one bse_build_block, in real flops with a
 * complex multiply-add counted as 8, over the unordered pairs of k stars the
 * build visits (a <= b, and k <= k' inside a star); rho and contract count
 * the k pairs the direct kernel computes (the seeds when bse_set_seeds is on):
 *   rho      = 8 (Nc^2 + Nv^2) sum_pairs n_ovl(k,k'),  n_ovl = #{(p', Q):
 *              p' in S_k', Q in S_q, p' + Q in S_k}
 *   contract = 8 sum_pairs (Nv^2 NG(q)^2 + Nc^2 Nv^2 NG(q))
 *   project  = 8 sum_tiles (|a| B sum_{j in b} n_o(j) + sum_{i in a} n_o(i) m_b)
 *   exchange = 8 (sum_i n_o(i) NG0 + sum_tiles m_a m_b NG0)
 * bse_build_work runs a counting kernel and blocks until it has finished.
 */
typedef struct {
    double rho, contract, project, exchange;
    int64_t k_pairs;       /* unordered k pairs of the direct term */
    int64_t overlap;       /* sum over the computed pairs of n_ovl */
    int64_t tiles;         /* star-pair tiles */
    int64_t seeds;         /* k pairs the direct kernel computes (all of them without seeds) */
    int64_t rotated;       /* k pairs rotated from their seeds (Eq. Wtrafo) */
    double rotate;         /* flops of the rotations: 16 B sum over both sides of the multiplet terms */
} bse_work;

int bse_build_work(bse_ctx* ctx, int32_t irrep, int32_t partner, bse_work* out);   /* partner: 0 block, 1 partner block */
/* the same for one bse_build_blocks call (arguments as there); the direct
 * term's pairs are counted once, the projections once per target */
int bse_build_blocks_work(bse_ctx* ctx, int32_t n, const int32_t* irrep, const int32_t* partner, bse_work* out);

/*
 * bse_stats: kernel launches of this library in the process so far, and,
 * when timing is on (bse_set_timing), the device time of the stages of the
 * last bse_build_block / bse_block_spectrum measured with CUDA events on the
 * context's stream.  bse_get_stats synchronises that stream.
 */
typedef struct {
    int64_t launches;           /* process-wide count of this library's kernel launches */
    int64_t direct_launches;    /* direct-term kernel launches of the last build */
    float ms_direct;            /* direct-term kernel(s) of the last build */
    float ms_project;           /* both projection stages of the last build */
    float ms_exchange;          /* exchange projection of the last build */
    float ms_eig;               /* dense eigensolver of the last spectrum */
    float ms_spectrum;          /* oscillator strengths and Im eps of the last spectrum */
    float ms_create;            /* wall time of bse_create */
    float ms_create_tables;     /* ... host tables (group, mesh, stars, characters, orbits) */
    float ms_create_upload;     /* ... device copies of the inputs and the look-up box */
    float ms_create_gamma;      /* ... band rotations (kernels, copy back, unitarity check) */
    float ms_create_wdiv;       /* ... head correction: host time to launch it (its kernels run behind the host work that follows) */
    float ms_basis;             /* wall time of the last basis construction (host, incl. upload) */
    int32_t solver;             /* eigensolver of the last spectrum: BSE_SOLVER_DENSE or BSE_SOLVER_TRIDIAG */
    float ms_reduce;            /* tridiagonal reduction kernel of the last spectrum (TRIDIAG), else 0 */
    float ms_rotate;            /* rotated direct-term blocks of the last build (part of ms_direct) */
    int32_t reduce_kind;        /* reduction of the last TRIDIAG spectrum: 0 block in shared memory, 1 blocked
                                   (panels) with the tensor-core panel update, 2 blocked with the double-float one,
                                   3 two-stage (band, then bulge chasing) */
    int32_t tc_pairs_per_cta;   /* k pairs per CTA (sharing one W(q)) of the last split-precision build, as tuned */
    int32_t pad_;
} bse_stats;

int bse_set_timing(bse_ctx* ctx, int32_t on);
int bse_get_stats(bse_ctx* ctx, bse_stats* out);

/*
 * bse_head_correction_noalloc - the head correction W^div of bse_create
 * (b = 0.005) for a lattice (host [9], row-major, columns a1 a2 a3), a
 * Gamma-centred mesh (host [3]) and a dielectric tensor (host [9]), written
 * to w_div_dev (device, one double) on the given stream, without allocating
 * any memory.  The paper has no counterpart; it exists for callers that
 * cannot allocate device memory where they need the value (a framework that
 * owns the device memory budget through its own pool, a latency-critical loop
 * that cannot afford the implicit synchronisation of cudaMalloc/cudaFree, a
 * plug-in handed only pre-allocated buffers).
 * The partial sums live in a fixed device array of 65536 doubles (512 KiB)
 * inside the library, held on every device that loads the library until the
 * process exits; meshes whose lattice sum needs more partial sums are
 * rejected with EINVAL.  The first call on a device looks up that array's
 * address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  All calls share the array and it keeps
 * the last call's contents; nothing in it has to start at zero.  Calls whose
 * work overlaps on the GPU (other streams, other host threads) race on it.
 * Returns once the work is enqueued.
 */
int bse_head_correction_noalloc(const double* lattice, const int32_t* mesh, const double* eps_inf,
                                double* w_div_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
