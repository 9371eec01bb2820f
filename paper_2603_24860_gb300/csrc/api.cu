// C ABI of the symmetry-reduced BSE block builder: context set-up, the
// star-pair tiling of the fused build + projection, and the block spectrum.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace bse {
const char* last_error();
}

static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

using namespace bse;

namespace {

// Device memory of a context comes from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the context's stream).  The pool keeps
// up to kPoolKeep bytes that contexts free for the next one, so creating a
// context per workload costs no driver allocation once the pool is warm.
constexpr uint64_t kPoolKeep = 64ull << 30;
thread_local cudaStream_t t_alloc_stream = nullptr;

struct AllocStream {   // stream the allocations of one API call are ordered on
    cudaStream_t prev;
    explicit AllocStream(cudaStream_t s) : prev(t_alloc_stream) { t_alloc_stream = s; }
    ~AllocStream() { t_alloc_stream = prev; }
};

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaStream_t st = nullptr;   // stream of the allocation (its free is ordered there)
};

int ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.n >= bytes) return BSE_OK;
    if (b.p) cudaFreeAsync(b.p, b.st);
    b.p = nullptr;
    b.n = 0;
    cudaError_t e = cudaMallocAsync(&b.p, bytes, t_alloc_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(BSE_ENOMEM, "cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
    }
    b.n = bytes;
    b.st = t_alloc_stream;
    return BSE_OK;
}

void release(DevBuf& b) {
    if (b.p) cudaFreeAsync(b.p, b.st);
    b.p = nullptr;
    b.n = 0;
}

int keep_pool_memory() {
    int dev = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    BSE_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t keep = kPoolKeep;
    BSE_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    return BSE_OK;
}

template <class T>
int upload(DevBuf& b, const T* src, size_t count, cudaStream_t st) {
    BSE_TRY(ensure(b, sizeof(T) * count));
    if (count) BSE_CUDA(cudaMemcpyAsync(b.p, src, sizeof(T) * count, cudaMemcpyDefault, st));
    return BSE_OK;
}

struct IrrepDev {
    bool ready = false;
    Basis host;
    DevBuf col_orbit, col_off, coef;
    DevBuf coef_df;   // coef in double-float, for the projection of FP32 tiles
};

}  // namespace

struct bse_ctx {
    Tables t;
    cudaStream_t stream = nullptr;
    DevSys S{};
    std::vector<int32_t> npw, ng, gk, gq;
    DevBuf coef, eps, w, dgk, dgq, dnpw, dng, kidx, box, rk, tau, rotk, vbar;
    DevBuf orbit_off, members, member_loc;
    std::vector<IrrepDev> irr;
    std::vector<int64_t> block_dim;
    struct PartnerDev {
        bool ready = false;
        int d = 0;
        IrrepDev part[3];   // partner 1 basis and its transfers P_i1 U_1
    };
    std::vector<PartnerDev> partner;
    // partner data of each irrep, made on first use (ensure_pmat): dim_mu / d_mu
    // for partner-capable irreps (else 0), the irrep matrices [s][d][d] and d
    mutable std::vector<int64_t> partner_dim;
    mutable std::vector<std::vector<double>> pgam;
    mutable std::vector<int> pgam_d;
    mutable std::vector<char> pready;
    std::vector<cplx> ptrace;   // Tr Gamma~(s) of the product space, for Tr P_11
    int ng0 = 0;
    mutable double w_div = 0.0;        // host copy of W^div, valid when wdiv_host_ok
    mutable bool wdiv_host_ok = false;
    double spin = 2.0;
    DevBuf P;            // exchange vectors [N][ng0]
    DevBuf Pt;           // projected exchange vectors scaled by v^1/2, double-float (mixed builds)
    bool P_ready = false;
    DevBuf B;            // dipoles [N]
    bool B_ready = false;
    DevBuf de;           // eps_c - eps_v per product index (FP64)
    DevBuf coef32, w32;  // FP32 copies for the FP32 build, made on first use
    bool narrow_ready = false;
    DevBuf wemb;         // split-precision W(q) embeddings for the tensor-core build
    DevBuf wexp;         // their per-q scale exponents
    DevBuf lzScratch;    // Lanczos vectors, T_m and its eigenvectors
    int wemb_ngp = 0;
    int wemb_fp16 = -1;  // element type of wemb (1 fp16, 0 bf16)
    DevBuf groups, status;
    DevBuf tcinst, tcq;  // the tensor-core launch's system and its work-queue counter
    DevBuf dinst;        // the context's system as a direct-kernel instance
    // band rotations kept on the device for the rotated direct-term blocks (Eq. Wtrafo)
    DevBuf gam, gam32, gkoff, gboff, mfirst, msize;
    bool seeds = true;   // compute one k pair per symmetry orbit and rotate the rest
    DevBuf rots;
    DevBuf rtiles, rmeta;   // device enumeration of the rotated pairs: tile records, per-member arrays
    DevBuf rtab_buf;        // group and star tables it reads (made on first use)
    RotTables rtab{};
    bool rtab_ready = false;
    DevBuf lossScratch;
    DevBuf wsym;         // orbit sum of W^div: per-column arrays
    DevBuf wdivDev;      // W^div on the device (one double), read by the kernels that need it
    int32_t solver_mode = BSE_SOLVER_AUTO;
    long wait_polls = -1;   // polls of every bounded device wait (negative: the kernels' defaults)
    DevBuf triScratch, triSmall;   // tridiagonal path: scratch; gram [9], weight sum, error flag
    // scratch (library-owned, grow-only)
    DevBuf arenaX, arenaY, Pmu, tasks, tiles, pairs, eigA, eigWork, info, Bmu, wpart, wsum, counter;
    cusolverDnHandle_t solver = nullptr;
    // measurement
    bool timing = false;
    cudaEvent_t ev[10] = {};
    bse_stats stats{};
};

namespace {

// std::allocator whose resize leaves trivially constructible elements
// uninitialised: the planner fills the task lists in parallel afterwards
template <class T>
struct NoInit : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInit<U>;
    };
    NoInit() = default;
    template <class U>
    NoInit(const NoInit<U>&) {}
    template <class U>
    void construct(U* p) noexcept {
        ::new ((void*)p) U;
    }
    template <class U, class... A>
    void construct(U* p, A&&... args) {
        ::new ((void*)p) U(std::forward<A>(args)...);
    }
};

// star-pair tiles shared by one or more target bases (irrep blocks or partner
// blocks), grouped into batches whose X and Y arenas fit a budget.  X (the
// direct term on the product basis of a star pair) does not depend on the
// target, so every target of a batch projects the same X tiles.
struct Batch {
    std::vector<PairTask> tasks;          // k pairs the direct kernel computes (seeds when symmetry is used)
    std::vector<RotTask, NoInit<RotTask>> rots;   // k pairs rotated from their seed (Eq. Wtrafo), host list
    std::vector<RotTile> rtiles;          // or: the tiles whose rotated pairs the device enumerates,
    std::vector<int> rmeta;               // their per-member arrays (jr, then gop, then seedpre)
    int64_t npairs = 0, nrots = 0;        // the pairs of those tiles and the rotated ones
    std::vector<TileTask> tiles;          // all targets' tiles, concatenated
    std::vector<int> tile_off;            // [targets + 1] range of each target in tiles
    size_t xbytes = 0;
    std::vector<size_t> ybytes;           // per target
    std::vector<int64_t> max_rows, max_ca, max_cb;   // per target
};

// Budget of each tile arena (bytes of FP64 tiles; the FP32 builds use half).
// BSE_ARENA_MB fixes it; otherwise it is a sixth of the device's free memory,
// between 2 and 32 GiB, so that the tiles of a workload such as the 12x12x12
// mesh's T1u block fit one batch (one launch of each kernel of the build)
// whenever the device has room.
size_t arena_budget() {
    const char* env = std::getenv("BSE_ARENA_MB");
    if (env) return (size_t)std::atoll(env) << 20;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return (size_t)2048 << 20;
    }
    return std::min<size_t>(std::max<size_t>(fr / 6, (size_t)2 << 30), (size_t)32 << 30);
}

// Seeds of a star-pair tile (a, b) (Eq. Wtrafo): every k pair (k, k') is
// (s k0, s k'_r)-equivalent to a pair with k0 = star a's representative and
// k'_r the representative (lowest k) of the orbit of k' under the little
// group of k0.  rep[j], gop[j] for the members j of star b: that
// representative and the first operation of the little group lg (ascending)
// taking k'_j to it.
static void little_orbits(const Tables& t, const std::vector<int>& lg, int b, int* rep, int* gop) {
    const auto& sb = t.stars[b];
    for (size_t j = 0; j < sb.size(); ++j) {
        rep[j] = -1;
        gop[j] = -1;
        const int kp = sb[j];
        for (int g : lg) {
            const int x = t.rotk[(size_t)g * t.nk + kp];
            if (rep[j] < 0 || x < rep[j]) {
                rep[j] = x;
                gop[j] = g;
            }
        }
    }
}

// Batches of star-pair tiles (a <= b over the stars some target uses) under
// the arena budget, with every target's tiles and the k pairs of each tile:
// the seeds the direct kernel computes and the pairs rotated from them.  The
// tiles are placed in one sequential pass (cheap); the k pairs, about N_k^2/2
// of them, are counted and then written by the host thread pool, tile by
// tile, at offsets from a prefix sum, in the same order as a sequential loop.
int plan_batches(const Tables& t, const std::vector<const Basis*>& bases, size_t budget, std::vector<Batch>& out,
                 bool seeds = false, bool host_rots = true) {
    out.clear();
    std::vector<int> inv(t.nops, -1);
    for (int a = 0; a < t.nops; ++a)
        for (int b = 0; b < t.nops; ++b)
            if (t.mult[(size_t)a * t.nops + b] == t.identity) inv[a] = b;
    const size_t nt = bases.size();
    auto ncols = [&](size_t i, int a) { return bases[i]->star_col[a + 1] - bases[i]->star_col[a]; };
    std::vector<int> act;
    for (size_t a = 0; a < t.stars.size(); ++a)
        for (size_t i = 0; i < nt; ++i)
            if (ncols(i, (int)a) > 0) {
                act.push_back((int)a);
                break;
            }
    const int B = t.B;
    // little group of each used star's representative (ascending operations)
    std::vector<std::vector<int>> lg(t.stars.size());
    if (seeds)
        for (int a : act) {
            const int k0 = t.stars[a][0];
            for (int g = 0; g < t.nops; ++g)
                if (t.rotk[(size_t)g * t.nk + k0] == k0) lg[a].push_back(g);
        }
    struct Tile {
        int a, b, batch;
        int64_t xoff, rows;
        int64_t seeds = 0, pairs = 0, task_off = 0, rot_off = 0;
        int64_t rep_off = 0;   // its members' entries in rep / gop
    };
    std::vector<int> rep, gop;   // little-orbit representative of each member of star b, and the operation
    std::vector<Tile> tiles;
    std::vector<std::vector<TileTask>> per(nt);
    Batch cur;
    int nb = 0;
    auto reset = [&]() {
        cur = Batch();
        cur.ybytes.assign(nt, 0);
        cur.max_rows.assign(nt, 0);
        cur.max_ca.assign(nt, 0);
        cur.max_cb.assign(nt, 0);
        for (auto& v : per) v.clear();
    };
    auto flush = [&]() {
        cur.tile_off.assign(1, 0);
        for (size_t i = 0; i < nt; ++i) {
            cur.tiles.insert(cur.tiles.end(), per[i].begin(), per[i].end());
            cur.tile_off.push_back((int)cur.tiles.size());
        }
        out.push_back(std::move(cur));
        ++nb;
    };
    reset();
    bool any = false;   // the current batch has a tile
    for (size_t iA = 0; iA < act.size(); ++iA)
        for (size_t iB = iA; iB < act.size(); ++iB) {
            const int a = act[iA], b = act[iB];
            bool used = false;
            for (size_t i = 0; i < nt; ++i) used = used || (ncols(i, a) > 0 && ncols(i, b) > 0);
            if (!used) continue;
            const int64_t rows = (int64_t)t.stars[a].size() * B, cols = (int64_t)t.stars[b].size() * B;
            const size_t xs = sizeof(double2) * rows * cols;
            bool full = any && cur.xbytes + xs > budget;
            for (size_t i = 0; i < nt && !full; ++i)
                full = any && ncols(i, a) > 0 && cur.ybytes[i] + sizeof(double2) * rows * ncols(i, b) > budget;
            if (full) {
                flush();
                reset();
            }
            const int64_t xoff = (int64_t)(cur.xbytes / sizeof(double2));
            for (size_t i = 0; i < nt; ++i) {
                const int64_t ma = ncols(i, a), mb = ncols(i, b);
                if (ma == 0 || mb == 0) continue;
                TileTask tt;
                tt.xoff = xoff;
                tt.yoff = (int64_t)(cur.ybytes[i] / sizeof(double2));
                tt.rows = (int32_t)rows;
                tt.cols = (int32_t)cols;
                tt.star_a = a;
                tt.star_b = b;
                tt.ca0 = bases[i]->star_col[a];
                tt.ca1 = bases[i]->star_col[a + 1];
                tt.cb0 = bases[i]->star_col[b];
                tt.cb1 = bases[i]->star_col[b + 1];
                per[i].push_back(tt);
                cur.ybytes[i] += sizeof(double2) * rows * mb;
                cur.max_rows[i] = std::max(cur.max_rows[i], rows);
                cur.max_ca[i] = std::max(cur.max_ca[i], ma);
                cur.max_cb[i] = std::max(cur.max_cb[i], mb);
            }
            Tile tl;
            tl.a = a;
            tl.b = b;
            tl.batch = nb;
            tl.xoff = xoff;
            tl.rows = rows;
            const int64_t na = (int64_t)t.stars[a].size(), nbm = (int64_t)t.stars[b].size();
            tl.pairs = a == b ? na * (na + 1) / 2 : na * nbm;
            tl.rep_off = (int64_t)rep.size();
            if (seeds) {
                rep.resize(rep.size() + nbm);
                gop.resize(gop.size() + nbm);
            }
            tiles.push_back(tl);
            cur.xbytes += xs;
            any = true;
        }
    if (any) flush();
    // k pairs: seeds per tile (the members of star b that are their own
    // little-orbit representative, paired with k0), offsets, then the lists
    const int ntl = (int)tiles.size();
    for (Tile& tl : tiles) {   // small: |star b| x |little group| per tile
        if (seeds) {
            int* rp = rep.data() + tl.rep_off;
            little_orbits(t, lg[tl.a], tl.b, rp, gop.data() + tl.rep_off);
            const auto& sb = t.stars[tl.b];
            for (size_t j = 0; j < sb.size(); ++j) tl.seeds += rp[j] == sb[j];
        } else {
            tl.seeds = tl.pairs;
        }
    }
    {
        std::vector<int64_t> nt_task(out.size(), 0), nt_rot(out.size(), 0);
        for (Tile& tl : tiles) {
            tl.task_off = nt_task[tl.batch];
            tl.rot_off = nt_rot[tl.batch];
            nt_task[tl.batch] += tl.seeds;
            nt_rot[tl.batch] += tl.pairs - tl.seeds;
        }
        for (size_t q = 0; q < out.size(); ++q) {
            out[q].tasks.resize((size_t)nt_task[q]);
            out[q].nrots = nt_rot[q];
            if (host_rots || !seeds) out[q].rots.resize((size_t)nt_rot[q]);
        }
    }
    const bool dev_rots = seeds && !host_rots;
    if (dev_rots)   // the device enumerates the rotated pairs: tile records and per-member arrays
        for (size_t q = 0; q < out.size(); ++q) {
            Batch& bt = out[q];
            std::vector<int> jr, go, pre;
            for (const Tile& tl : tiles) {
                if (tl.batch != (int)q || tl.pairs == tl.seeds) continue;
                const auto& sb = t.stars[tl.b];
                const int* rp = rep.data() + tl.rep_off;
                const int* gp = gop.data() + tl.rep_off;
                RotTile rt;
                rt.xoff = tl.xoff;
                rt.pair_off = bt.npairs;
                rt.rot_off = tl.rot_off;
                rt.rows = (int32_t)tl.rows;
                rt.a = tl.a;
                rt.b = tl.b;
                rt.tri = tl.a == tl.b;
                rt.seeds = (int32_t)tl.seeds;
                rt.rep_off = (int32_t)jr.size();
                int before = 0;
                for (size_t j = 0; j < sb.size(); ++j) {
                    jr.push_back(t.pos_in_star[rp[j]]);
                    go.push_back(gp[j]);
                    pre.push_back(before);
                    before += rp[j] == sb[j];
                }
                bt.rtiles.push_back(rt);
                bt.npairs += tl.pairs;
            }
            bt.rmeta = jr;
            bt.rmeta.insert(bt.rmeta.end(), go.begin(), go.end());
            bt.rmeta.insert(bt.rmeta.end(), pre.begin(), pre.end());
        }
    std::vector<char> bad(ntl, 0);
    auto fill = [&](int q) {
        const Tile& tl = tiles[q];
        Batch& bt = out[tl.batch];
        const int a = tl.a, b = tl.b;
        const int64_t xoff = tl.xoff, rows = tl.rows;
        const auto& sa = t.stars[a];
        const auto& sb = t.stars[b];
        const int k0 = sa[0];
        PairTask* pt = bt.tasks.data() + tl.task_off;
        int64_t ntask = 0, nrot = 0;
        const int* rp = seeds ? rep.data() + tl.rep_off : nullptr;
        const int* gp = seeds ? gop.data() + tl.rep_off : nullptr;
        if (dev_rots) {   // seeds only: (k0, k'_j) for j its own little-orbit representative
            for (size_t j = 0; j < sb.size(); ++j) {
                if (rp[j] != sb[j]) continue;
                if (ntask >= tl.seeds) {
                    bad[q] = 2;
                    return;
                }
                PairTask& p = pt[ntask++];
                p.k = k0;
                p.kp = sb[j];
                p.row0 = 0;
                p.col0 = (int32_t)(j * B);
                p.xoff = xoff;
                p.ld = (int32_t)rows;
                p.flags = (a == b && j > 0) ? 1 : 0;
            }
            if (ntask != tl.seeds) bad[q] = 2;
            return;
        }
        RotTask* rt = bt.rots.data() + tl.rot_off;
        for (size_t i = 0; i < sa.size(); ++i)
            for (size_t j = (a == b ? i : 0); j < sb.size(); ++j) {
                if (seeds) {
                    const int k = sa[i], kp = sb[j];
                    const int s1 = inv[t.s_k[k]];   // takes k to k0
                    const int jpp = t.pos_in_star[t.rotk[(size_t)s1 * t.nk + kp]];
                    const int r = rp[jpp];
                    const int s = t.mult[(size_t)gp[jpp] * t.nops + s1];
                    if (t.rotk[(size_t)s * t.nk + k] != k0 || t.rotk[(size_t)s * t.nk + kp] != r) {
                        bad[q] = 1;
                        return;
                    }
                    const int jr = t.pos_in_star[r];
                    if (!(i == 0 && (int)j == jr)) {
                        if (tl.rot_off + nrot >= tl.rot_off + (tl.pairs - tl.seeds)) {
                            bad[q] = 2;
                            return;
                        }
                        RotTask& o = rt[nrot++];
                        o.src = xoff + (int64_t)jr * B * rows;
                        o.dst = xoff + (int64_t)j * B * rows + (int64_t)i * B;
                        o.dstm = xoff + (int64_t)i * B * rows + (int64_t)j * B;
                        o.k = k;
                        o.kp = kp;
                        o.s = s;
                        o.ld = (int32_t)rows;
                        o.flags = (a == b && j > i) ? 1 : 0;
                        o.pad = 0;
                        continue;
                    }
                }
                if (ntask >= tl.seeds) {
                    bad[q] = 2;
                    return;
                }
                PairTask& p = pt[ntask++];
                p.k = sa[i];
                p.kp = sb[j];
                p.row0 = (int32_t)(i * B);
                p.col0 = (int32_t)(j * B);
                p.xoff = xoff;
                p.ld = (int32_t)rows;
                p.flags = (a == b && j > i) ? 1 : 0;
            }
        if (ntask != tl.seeds || nrot != tl.pairs - tl.seeds) bad[q] = 2;
    };
    if (dev_rots) {
        for (int q = 0; q < ntl; ++q) fill(q);
    } else {   // every k pair on the host: the host thread pool, largest tiles first
        std::vector<double> cost(ntl);
        for (int q = 0; q < ntl; ++q) cost[q] = (double)tiles[q].pairs;
        host_parallel_for(ntl, fill, &cost);
    }
    for (int q = 0; q < ntl; ++q) {
        if (bad[q] == 1) return fail(BSE_ESYMM, "seed of a k pair of star pair (%d, %d) not found", tiles[q].a, tiles[q].b);
        if (bad[q] == 2)
            return fail(BSE_ESYMM, "star pair (%d, %d): seeds are not the own little-orbit representatives",
                        tiles[q].a, tiles[q].b);
    }
    return BSE_OK;
}

}  // namespace

static DevBasis dev_basis_of(bse_ctx* c, IrrepDev& d) {
    DevBasis b;
    b.dim = d.host.dim;
    b.col_orbit = (const int*)d.col_orbit.p;
    b.col_off = (const int64_t*)d.col_off.p;
    b.coef = (const double2*)d.coef.p;
    b.coef_df = (const float4*)d.coef_df.p;
    b.orbit_off = (const int64_t*)c->orbit_off.p;
    b.members = (const int64_t*)c->members.p;
    b.member_loc = (const int*)c->member_loc.p;
    return b;
}

static DevBasis dev_basis(bse_ctx* c, int mu) { return dev_basis_of(c, c->irr[mu]); }

static int upload_basis(bse_ctx* c, IrrepDev& d) {
    BSE_TRY(upload(d.col_orbit, d.host.col_orbit.data(), d.host.col_orbit.size(), c->stream));
    BSE_TRY(upload(d.col_off, d.host.col_off.data(), d.host.col_off.size(), c->stream));
    BSE_TRY(upload(d.coef, reinterpret_cast<const double2*>(d.host.coef.data()), d.host.coef.size(), c->stream));
    BSE_TRY(ensure(d.coef_df, sizeof(float4) * d.host.coef.size()));
    BSE_TRY(launch_to_df((const double2*)d.coef.p, (float4*)d.coef_df.p, (int64_t)d.host.coef.size(), c->stream));
    BSE_CUDA(cudaStreamSynchronize(c->stream));
    d.ready = true;
    return BSE_OK;
}

// irrep matrices of irrep mu (when it has them) and its partner dimension
// Tr P_11 = d/|S| sum_s Gamma_mu(s)_11 Tr Gamma~(s), made once
static int ensure_pmat(const bse_ctx* c, int mu) {
    if (c->pready[mu]) return BSE_OK;
    const Tables& t = c->t;
    int d = 0;
    std::vector<double> gam;
    if (partner_matrices(t, mu, d, gam) != BSE_OK) {   // no irrep matrices: no partner block
        clear_error();
        c->pready[mu] = 1;
        return BSE_OK;
    }
    cplx a = 0;
    for (int s = 0; s < t.nops; ++s) a += gam[(size_t)s * d * d] * c->ptrace[s];
    const double dd = a.real() * d / t.nops;
    const long r = std::lround(dd);
    if (std::fabs(dd - r) > 1e-6 || r * d != c->block_dim[mu])
        return fail(BSE_ESYMM, "Tr P_11 of irrep %d = %.9f is not dim/d", mu, dd);
    c->pgam[mu] = std::move(gam);
    c->pgam_d[mu] = d;
    c->partner_dim[mu] = r;
    c->pready[mu] = 1;
    return BSE_OK;
}

// partner 1 of an irrep: canonical basis of the range of P_11 and its
// transfers U_i = P_i1 U_1
static int ensure_partner(bse_ctx* c, int mu) {
    if (mu < 0 || mu >= c->t.n_irreps) return fail(BSE_EINVAL, "irrep %d out of range [0, %d)", mu, c->t.n_irreps);
    auto& pd = c->partner[mu];
    if (pd.ready) return BSE_OK;
    BSE_TRY(ensure_pmat(c, mu));
    const double t0 = now_ms();
    const int d = c->pgam_d[mu];
    if (d == 0) return fail(BSE_EUNSUPPORTED, "irrep %d has no irrep matrices for a partner block", mu);
    const std::vector<double>& gam = c->pgam[mu];
    const int G = c->t.nops;
    auto weights = [&](int i, int j) {
        std::vector<double> w(G);
        for (int s = 0; s < G; ++s) w[s] = (double)d / G * gam[((size_t)s * d + i) * d + j];
        return w;
    };
    BSE_TRY(build_basis_weighted(c->t, weights(0, 0), pd.part[0].host));
    if (pd.part[0].host.dim != c->partner_dim[mu])
        return fail(BSE_ESYMM, "irrep %d: partner basis has %lld vectors but Tr P_11 = %lld", mu,
                    (long long)pd.part[0].host.dim, (long long)c->partner_dim[mu]);
    {
        std::vector<std::vector<double>> ws;
        std::vector<Basis*> outs;
        for (int i = 1; i < d; ++i) {
            ws.push_back(weights(i, 0));
            outs.push_back(&pd.part[i].host);
        }
        if (d > 1) BSE_TRY(transfer_bases(c->t, pd.part[0].host, ws, outs));
    }
    for (int i = 0; i < d; ++i) BSE_TRY(upload_basis(c, pd.part[i]));
    pd.d = d;
    pd.ready = true;
    c->stats.ms_basis = (float)(now_ms() - t0);
    return BSE_OK;
}

static int ensure_basis(bse_ctx* c, int mu) {
    if (mu < 0 || mu >= c->t.n_irreps) return fail(BSE_EINVAL, "irrep %d out of range [0, %d)", mu, c->t.n_irreps);
    IrrepDev& d = c->irr[mu];
    if (d.ready) return BSE_OK;
    const double t0 = now_ms();
    BSE_TRY(build_basis(c->t, mu, d.host));
    if (d.host.dim != c->block_dim[mu])
        return fail(BSE_ESYMM, "irrep %d: orthonormal basis has %lld vectors but Tr P = %lld", mu,
                    (long long)d.host.dim, (long long)c->block_dim[mu]);
    BSE_TRY(upload_basis(c, d));
    c->stats.ms_basis = (float)(now_ms() - t0);
    return BSE_OK;
}

static int ensure_exchange_vectors(bse_ctx* c) {
    if (c->P_ready) return BSE_OK;
    const int nk = c->t.nk;
    std::vector<int32_t> kk(nk);
    for (int k = 0; k < nk; ++k) kk[k] = k;
    BSE_TRY(upload(c->pairs, kk.data(), kk.size(), c->stream));
    BSE_TRY(ensure(c->P, sizeof(double2) * (size_t)c->t.N * c->ng0));
    BSE_TRY(launch_pairdens(c->S, (const int*)c->pairs.p, (const int*)c->pairs.p, nk, BSE_BANDS_CV, 1,
                            (double2*)c->P.p, c->stream));
    BSE_CUDA(cudaStreamSynchronize(c->stream));
    c->P_ready = true;
    return BSE_OK;
}

static int ensure_dipoles(bse_ctx* c) {
    if (c->B_ready) return BSE_OK;
    BSE_TRY(ensure(c->B, sizeof(double2) * (size_t)c->t.N));
    BSE_TRY(launch_dipoles(c->S, (double2*)c->B.p, c->stream));
    c->B_ready = true;
    return BSE_OK;
}

static int ensure_wemb(bse_ctx* c, int ngp, int fp16) {
    if (c->wemb_ngp == ngp && c->wemb_fp16 == fp16) return BSE_OK;
    BSE_TRY(ensure(c->wemb, sizeof(uint16_t) * (size_t)c->t.nk * 2 * 128 * 2 * ngp));
    BSE_TRY(ensure(c->wexp, sizeof(int) * (size_t)c->t.nk));
    BSE_TRY(launch_wemb(c->S, ngp, fp16, c->wemb.p, (int*)c->wexp.p, c->stream));
    c->wemb_ngp = ngp;
    c->wemb_fp16 = fp16;
    return BSE_OK;
}

static int ensure_narrow(bse_ctx* c) {
    if (c->narrow_ready) return BSE_OK;
    const int64_t nc = (int64_t)c->t.nk * c->t.nb * c->S.npw_max;
    const int64_t nw = (int64_t)c->t.nk * c->S.ng_max * c->S.ng_max;
    BSE_TRY(ensure(c->coef32, sizeof(float2) * (size_t)nc));
    BSE_TRY(ensure(c->w32, sizeof(float2) * (size_t)nw));
    BSE_TRY(launch_narrow(c->S.coef, (float2*)c->coef32.p, nc, c->stream));
    BSE_TRY(launch_narrow(c->S.w, (float2*)c->w32.p, nw, c->stream));
    const int64_t ng = (int64_t)c->t.nops * c->t.gam_per_s;
    BSE_TRY(ensure(c->gam32, sizeof(float2) * (size_t)std::max<int64_t>(ng, 1)));
    BSE_TRY(launch_narrow((const double2*)c->gam.p, (float2*)c->gam32.p, ng, c->stream));
    c->narrow_ready = true;
    return BSE_OK;
}

// H00 = (1/sqrt(4 pi)) int dOmega 1/(q^T L q): closed form when L is isotropic,
// otherwise Gauss-Legendre in cos(theta) times a periodic trapezoid in phi.
static double h00(const double* L) {
    bool iso = true;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if ((i == j && L[3 * i + j] != L[0]) || (i != j && L[3 * i + j] != 0.0)) iso = false;
    if (iso) return std::sqrt(4.0 * M_PI) / L[0];
    const int nt = 96, np = 192;
    std::vector<double> x(nt), wt(nt);
    for (int i = 0; i < nt; ++i) {   // Newton iteration on P_nt
        double z = std::cos(M_PI * (i + 0.75) / (nt + 0.5)), pp = 0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= nt; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = nt * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
    double acc = 0.0;
    for (int i = 0; i < nt; ++i) {
        double ct = x[i], st = std::sqrt(1.0 - ct * ct);
        for (int j = 0; j < np; ++j) {
            double ph = 2.0 * M_PI * j / np;
            double n[3] = {st * std::cos(ph), st * std::sin(ph), ct};
            double q = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) q += n[a] * L[3 * a + b] * n[b];
            acc += wt[i] * (2.0 * M_PI / np) / q;
        }
    }
    return acc / std::sqrt(4.0 * M_PI);
}

namespace bse {
// H00 for callers outside this file
double head_h00(const double* L) { return h00(L); }
}  // namespace bse

static int compute_wdiv(bse_ctx* c, const double* L) {
    const double b = 0.005;
    const double qmax = std::sqrt(-std::log(b) / b);
    const double vbz = 8.0 * M_PI * M_PI * M_PI / c->t.v_uc;
    const double delta = std::cbrt(vbz / c->t.nk);
    int64_t np = wdiv_partials(c->t.lattice, c->t.n, qmax, delta);
    BSE_TRY(ensure(c->wpart, sizeof(double) * (size_t)np));
    BSE_TRY(ensure(c->wsum, sizeof(double)));
    double rl[18];
    std::memcpy(rl, c->t.recip, sizeof(double) * 9);
    std::memcpy(rl + 9, c->t.lattice, sizeof(double) * 9);
    // the point group on the integer coordinates X of Q = sum_j X_j b_j / n_j:
    // M = D rk D^-1 (rk = R^-T on fractional reciprocal coordinates, D = diag(n));
    // the sum runs over orbits when every M is integral and L is invariant
    std::vector<int> Mx((size_t)9 * c->t.nops);
    bool sym = c->t.nops <= 48;
    for (int s = 0; s < c->t.nops && sym; ++s)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const long num = (long)c->t.rk[9 * s + 3 * i + j] * c->t.n[i];
                if (num % c->t.n[j] != 0) sym = false;
                Mx[9 * s + 3 * i + j] = (int)(num / c->t.n[j]);
            }
    double lnorm = 0.0;
    for (int i = 0; i < 9; ++i) lnorm = std::max(lnorm, std::fabs(L[i]));
    for (int s = 0; s < c->t.nops && sym; ++s) {
        const double* R = &c->t.cart[9 * s];
        for (int i = 0; i < 3 && sym; ++i)
            for (int j = 0; j < 3 && sym; ++j) {
                double v = 0.0;   // (R L R^T)_ij
                for (int a = 0; a < 3; ++a)
                    for (int d = 0; d < 3; ++d) v += R[3 * i + a] * L[3 * a + d] * R[3 * j + d];
                if (std::fabs(v - L[3 * i + j]) > 1e-12 * lnorm) sym = false;
            }
    }
    WdivScratch ws;
    if (sym) {
        BSE_TRY(ensure(c->wsym, wdiv_sym_bytes(c->t.lattice, c->t.n, qmax, delta)));
        ws.base = c->wsym.p;
    }
    BSE_TRY(ensure(c->wdivDev, sizeof(double)));
    BSE_TRY(launch_wdiv(rl, c->t.n, L, b, qmax, delta, (double*)c->wpart.p, np, (double*)c->wsum.p, c->stream,
                        sym ? c->t.nops : 0, sym ? Mx.data() : nullptr, sym ? &ws : nullptr));
    // W^div = integral / (2 pi^2) - 4 pi / (N_k V) sum, left on the device: the
    // sum runs behind the host work that follows (the basis of the first build)
    const double integral = M_PI * h00(L) / std::sqrt(b) * std::erf(std::sqrt(b) * qmax);
    BSE_TRY(launch_wdiv_finalize((const double*)c->wsum.p, integral / (2.0 * M_PI * M_PI),
                                 4.0 * M_PI / (c->t.nk * c->t.v_uc), (double*)c->wdivDev.p, c->stream));
    c->wdiv_host_ok = false;
    return BSE_OK;
}

// the host copy of W^div (waits for its sum)
static int wdiv_host(const bse_ctx* c) {
    if (!c->wdiv_host_ok) {
        BSE_CUDA(cudaMemcpyAsync(&c->w_div, c->wdivDev.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        BSE_CUDA(cudaStreamSynchronize(c->stream));
        c->wdiv_host_ok = true;
    }
    return BSE_OK;
}

static int create_impl(bse_ctx* c, const bse_system* sys) {
    Tables& t = c->t;
    const double t0 = now_ms();
    if (sys->nv <= 0 || sys->nc <= 0) return fail(BSE_EINVAL, "nv and nc must be positive");
    if (sys->npw_max <= 0 || sys->npw_max > 32767 || sys->ng_max <= 0)
        return fail(BSE_EINVAL, "npw_max must be in 1..32767 and ng_max positive");
    if (!sys->npw || !sys->gk || !sys->coef || !sys->eps || !sys->ng || !sys->gq || !sys->w)
        return fail(BSE_EINVAL, "missing input array");
    if (sys->spin_factor <= 0) return fail(BSE_EINVAL, "spin_factor must be positive");
    t.nv = sys->nv;
    t.nc = sys->nc;
    t.nb = t.nv + t.nc;
    t.B = t.nv * t.nc;
    for (int i = 0; i < 3; ++i) t.n[i] = sys->mesh[i];
    BSE_TRY(build_group(t, sys));
    BSE_TRY(build_mesh(t));
    t.N = (int64_t)t.nk * t.B;
    c->spin = sys->spin_factor;
    const int nk = t.nk, nb = t.nb;
    c->npw.assign(sys->npw, sys->npw + nk);
    c->ng.assign(sys->ng, sys->ng + nk);
    c->gk.assign(sys->gk, sys->gk + (size_t)nk * sys->npw_max * 3);
    c->gq.assign(sys->gq, sys->gq + (size_t)nk * sys->ng_max * 3);
    for (int k = 0; k < nk; ++k) {
        if (c->npw[k] <= 0 || c->npw[k] > sys->npw_max) return fail(BSE_EINVAL, "npw[%d] out of range", k);
        if (c->ng[k] <= 0 || c->ng[k] > sys->ng_max) return fail(BSE_EINVAL, "ng[%d] out of range", k);
    }
    std::vector<double> eps_h((size_t)nk * nb);
    BSE_CUDA(cudaMemcpy(eps_h.data(), sys->eps, sizeof(double) * eps_h.size(), cudaMemcpyDefault));
    BSE_TRY(build_characters(t));
    BSE_TRY(build_multiplets_and_orbits(t, eps_h.data()));
    {
        std::vector<double> de((size_t)t.N);
        for (int k = 0; k < nk; ++k)
            for (int v = 0; v < t.nv; ++v)
                for (int cc = 0; cc < t.nc; ++cc)
                    de[((size_t)k * t.nv + v) * t.nc + cc] = eps_h[(size_t)k * nb + t.nv + cc] - eps_h[(size_t)k * nb + v];
        BSE_TRY(upload(c->de, de.data(), de.size(), c->stream));
        BSE_CUDA(cudaStreamSynchronize(c->stream));
    }
    const double t1 = now_ms();
    cudaStream_t st = c->stream;
    // device copies of the inputs
    BSE_TRY(upload(c->coef, reinterpret_cast<const double2*>(sys->coef), (size_t)nk * nb * sys->npw_max, st));
    BSE_TRY(upload(c->eps, sys->eps, (size_t)nk * nb, st));
    BSE_TRY(upload(c->w, reinterpret_cast<const double2*>(sys->w), (size_t)nk * sys->ng_max * sys->ng_max, st));
    BSE_TRY(upload(c->dgk, c->gk.data(), c->gk.size(), st));
    BSE_TRY(upload(c->dgq, c->gq.data(), c->gq.size(), st));
    BSE_TRY(upload(c->dnpw, c->npw.data(), c->npw.size(), st));
    BSE_TRY(upload(c->dng, c->ng.data(), c->ng.size(), st));
    BSE_TRY(upload(c->kidx, t.kidx.data(), t.kidx.size(), st));
    BSE_TRY(upload(c->rk, t.rk.data(), t.rk.size(), st));
    BSE_TRY(upload(c->tau, t.tau.data(), t.tau.size(), st));
    BSE_TRY(upload(c->rotk, t.rotk.data(), t.rotk.size(), st));
    // look-up box of the coset spheres
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (int k = 0; k < nk; ++k)
        for (int i = 0; i < c->npw[k]; ++i)
            for (int a = 0; a < 3; ++a) {
                int v = c->gk[((size_t)k * sys->npw_max + i) * 3 + a];
                lo[a] = std::min(lo[a], v);
                hi[a] = std::max(hi[a], v);
            }
    DevSys& S = c->S;
    int64_t bvol = 1;
    for (int a = 0; a < 3; ++a) {
        S.blo[a] = lo[a];
        S.bdim[a] = hi[a] - lo[a] + 1;
        bvol *= S.bdim[a];
    }
    S.bvol = bvol;
    std::vector<short> boxh((size_t)nk * bvol, (short)-1);
    for (int k = 0; k < nk; ++k)
        for (int i = 0; i < c->npw[k]; ++i) {
            const int* m = &c->gk[((size_t)k * sys->npw_max + i) * 3];
            int64_t pos = ((int64_t)(m[0] - lo[0]) * S.bdim[1] + (m[1] - lo[1])) * S.bdim[2] + (m[2] - lo[2]);
            short& slot = boxh[(size_t)k * bvol + pos];
            if (slot != -1) return fail(BSE_EINVAL, "plane wave repeated in the sphere of k=%d", k);
            slot = (short)i;
        }
    BSE_TRY(upload(c->box, boxh.data(), boxh.size(), st));
    // G = 0 in the sphere of q = 0 and the exchange Coulomb factors
    c->ng0 = c->ng[0];
    c->S.g0 = -1;
    std::vector<double> vb(c->ng0);
    for (int g = 0; g < c->ng0; ++g) {
        const int* m = &c->gq[(size_t)g * 3];
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) c->S.g0 = g;
        double G[3];
        for (int a = 0; a < 3; ++a) G[a] = t.recip[3 * a] * m[0] + t.recip[3 * a + 1] * m[1] + t.recip[3 * a + 2] * m[2];
        double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        vb[g] = g2 > 0 ? 4.0 * M_PI / g2 : 0.0;
    }
    if (c->S.g0 < 0) return fail(BSE_EINVAL, "the sphere of q = 0 lacks G = 0");
    BSE_TRY(upload(c->vbar, vb.data(), vb.size(), st));
    S.coef = (const double2*)c->coef.p;
    S.eps = (const double*)c->eps.p;
    S.w = (const double2*)c->w.p;
    S.gk = (const int*)c->dgk.p;
    S.gq = (const int*)c->dgq.p;
    S.npw = (const int*)c->dnpw.p;
    S.ng = (const int*)c->dng.p;
    S.kidx = (const int*)c->kidx.p;
    S.box = (const short*)c->box.p;
    S.n1 = t.n[0];
    S.n2 = t.n[1];
    S.n3 = t.n[2];
    S.nk = nk;
    S.nv = t.nv;
    S.nc = t.nc;
    S.nb = nb;
    S.npw_max = sys->npw_max;
    S.ng_max = sys->ng_max;
    S.inv_vol = 1.0 / (nk * t.v_uc);
    std::memcpy(S.recip, t.recip, sizeof(S.recip));
    double qn = std::sqrt(sys->qhat[0] * sys->qhat[0] + sys->qhat[1] * sys->qhat[1] + sys->qhat[2] * sys->qhat[2]);
    if (!(qn > 0)) return fail(BSE_EINVAL, "qhat must be nonzero");
    for (int a = 0; a < 3; ++a) S.qhat[a] = sys->qhat[a] / qn;
    S.v_uc = t.v_uc;
    S.scissor = sys->scissor;
    BSE_CUDA(cudaStreamSynchronize(st));
    const double t2 = now_ms();
    // band rotations Gamma(s) on the device
    std::vector<int32_t> ent;
    ent.reserve((size_t)t.gam_per_s * 3);
    for (int k = 0; k < nk; ++k) {
        for (auto* ms : {&t.vmult[k], &t.cmult[k]})
            for (auto& m : *ms)
                for (int a = 0; a < m.second; ++a)
                    for (int b = 0; b < m.second; ++b) {
                        ent.push_back(k);
                        ent.push_back(m.first + a);
                        ent.push_back(m.first + b);
                    }
    }
    DevBuf perm, phase, dent, dgam;
    int rc = BSE_OK;
    do {
        size_t nmap = (size_t)t.nops * nk * sys->npw_max;
        if ((rc = ensure(perm, sizeof(int) * nmap)) != BSE_OK) break;
        if ((rc = ensure(phase, sizeof(double2) * nmap)) != BSE_OK) break;
        if ((rc = upload(dent, ent.data(), ent.size(), st)) != BSE_OK) break;
        if ((rc = ensure(dgam, sizeof(double2) * (size_t)t.nops * t.gam_per_s)) != BSE_OK) break;
        if ((rc = launch_rotmap(S, (const int*)c->rk.p, (const double*)c->tau.p, (const int*)c->rotk.p, t.nops,
                                (int*)perm.p, (double2*)phase.p, st)) != BSE_OK)
            break;
        if ((rc = launch_gamma(S, t.nops, (const int*)c->rotk.p, (const int*)perm.p, (const double2*)phase.p,
                               (const int*)dent.p, t.gam_per_s, (double2*)dgam.p, st)) != BSE_OK)
            break;
        t.gamma.resize((size_t)t.nops * t.gam_per_s);
        cudaError_t e = cudaMemcpyAsync(t.gamma.data(), dgam.p, sizeof(double2) * t.gamma.size(),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = fail(BSE_ECUDA, "band rotations: %s", cudaGetErrorString(e));
    } while (0);
    release(perm);
    release(phase);
    release(dent);
    if (rc != BSE_OK) release(dgam);
    BSE_TRY(rc);
    c->gam = dgam;   // kept for the rotated direct-term blocks
    {
        std::vector<int32_t> mf((size_t)nk * t.nb), ms((size_t)nk * t.nb);
        for (int k = 0; k < nk; ++k)
            for (auto* mm : {&t.vmult[k], &t.cmult[k]})
                for (auto& m : *mm)
                    for (int b = m.first; b < m.first + m.second; ++b) {
                        mf[(size_t)k * t.nb + b] = m.first;
                        ms[(size_t)k * t.nb + b] = m.second;
                    }
        BSE_TRY(upload(c->gkoff, t.gam_koff.data(), t.gam_koff.size(), st));
        BSE_TRY(upload(c->gboff, t.gam_boff.data(), t.gam_boff.size(), st));
        BSE_TRY(upload(c->mfirst, mf.data(), mf.size(), st));
        BSE_TRY(upload(c->msize, ms.data(), ms.size(), st));
        BSE_CUDA(cudaStreamSynchronize(st));
    }
    BSE_TRY(check_band_rotations(t));
    const double t3 = now_ms();
    // block dimensions from the trace formula dim_mu = d_mu/|S| sum_s chi_mu(s) Tr Gamma~(s)
    std::vector<cplx> trace(t.nops, 0.0);
    for (int s = 0; s < t.nops; ++s)
        for (int k = 0; k < nk; ++k) {
            if (t.rotk[(size_t)s * nk + k] != k) continue;
            cplx tv = 0, tc = 0;
            int64_t off = (int64_t)s * t.gam_per_s + t.gam_koff[k];
            for (auto& m : t.vmult[k]) {
                for (int a = 0; a < m.second; ++a) tv += t.gamma[off + a * m.second + a];
                off += (int64_t)m.second * m.second;
            }
            for (auto& m : t.cmult[k]) {
                for (int a = 0; a < m.second; ++a) tc += t.gamma[off + a * m.second + a];
                off += (int64_t)m.second * m.second;
            }
            trace[s] += tc * std::conj(tv);
        }
    c->block_dim.assign(t.n_irreps, 0);
    int64_t tot = 0;
    for (int mu = 0; mu < t.n_irreps; ++mu) {
        cplx a = 0;
        for (int s = 0; s < t.nops; ++s) a += (double)t.chi[(size_t)mu * t.nops + s] * trace[s];
        double d = a.real() * t.irrep_dim[mu] / t.nops;
        long r = std::lround(d);
        if (std::fabs(d - r) > 1e-6 || std::fabs(a.imag()) > 1e-6)
            return fail(BSE_ESYMM, "Tr P_%d = %.9f is not an integer", mu, d);
        c->block_dim[mu] = r;
        tot += r;
    }
    if (tot != t.N) return fail(BSE_ESYMM, "block dimensions sum to %lld, not N = %lld", (long long)tot, (long long)t.N);
    // irrep matrices and partner dimensions are made per irrep on first use
    c->ptrace = trace;
    c->partner_dim.assign(t.n_irreps, 0);
    c->pgam.assign(t.n_irreps, {});
    c->pgam_d.assign(t.n_irreps, 0);
    c->pready.assign(t.n_irreps, 0);
    c->partner.resize(t.n_irreps);
    // orbit tables on the device
    std::vector<int> loc(t.orbit_members.size());
    for (size_t i = 0; i < loc.size(); ++i) {
        int64_t I = t.orbit_members[i];
        int k = (int)(I / t.B);
        loc[i] = t.pos_in_star[k] * t.B + (int)(I % t.B);
    }
    BSE_TRY(upload(c->orbit_off, t.orbit_off.data(), t.orbit_off.size(), st));
    BSE_TRY(upload(c->members, t.orbit_members.data(), t.orbit_members.size(), st));
    BSE_TRY(upload(c->member_loc, loc.data(), loc.size(), st));
    c->irr.resize(t.n_irreps);
    const double t4 = now_ms();
    if (std::isnan(sys->w_div)) {
        BSE_TRY(compute_wdiv(c, sys->eps_inf));   // asynchronous: no wait here
    } else {
        c->w_div = sys->w_div;
        c->wdiv_host_ok = true;
        BSE_TRY(upload(c->wdivDev, &c->w_div, 1, st));
    }
    const double t5 = now_ms();
    c->stats.ms_create_tables = (float)(t1 - t0);
    c->stats.ms_create_upload = (float)(t2 - t1);
    c->stats.ms_create_gamma = (float)(t3 - t2);
    c->stats.ms_create_wdiv = (float)(t5 - t4);
    c->stats.ms_create = (float)(t5 - t0);
    return BSE_OK;
}

static void free_ctx(bse_ctx* c) {
    for (DevBuf* b : {&c->coef, &c->eps, &c->w, &c->dgk, &c->dgq, &c->dnpw, &c->dng, &c->kidx, &c->box, &c->rk,
                      &c->tau, &c->rotk, &c->vbar, &c->orbit_off, &c->members, &c->member_loc, &c->P, &c->B,
                      &c->arenaX, &c->arenaY, &c->Pmu, &c->Pt, &c->tasks, &c->tiles, &c->pairs, &c->eigA, &c->eigWork,
                      &c->info, &c->Bmu, &c->wpart, &c->wsum, &c->de, &c->coef32, &c->w32, &c->wemb, &c->wexp, &c->groups, &c->status, &c->tcinst, &c->tcq,
                      &c->triScratch, &c->triSmall, &c->dinst,
                      &c->gam, &c->gam32, &c->gkoff, &c->gboff, &c->mfirst, &c->msize, &c->rots, &c->rtiles, &c->rmeta, &c->rtab_buf,
                      &c->lossScratch, &c->wsym, &c->wdivDev, &c->lzScratch})
        release(*b);
    for (auto& d : c->irr) {
        release(d.col_orbit);
        release(d.col_off);
        release(d.coef);
        release(d.coef_df);
    }
    for (auto& p : c->partner)
        for (auto& d : p.part) {
            release(d.col_orbit);
            release(d.col_off);
            release(d.coef);
            release(d.coef_df);
        }
    if (c->solver) cusolverDnDestroy(c->solver);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    release(c->counter);
    delete c;
}

// the context's band rotations as a rotation-kernel system
static RotSys rot_sys(bse_ctx* c, int p32) {
    RotSys r;
    r.gam = p32 ? c->gam32.p : c->gam.p;
    r.koff = (const int64_t*)c->gkoff.p;
    r.boff = (const int64_t*)c->gboff.p;
    r.mfirst = (const int*)c->mfirst.p;
    r.msize = (const int*)c->msize.p;
    r.gps = c->t.gam_per_s;
    r.nk = c->t.nk;
    r.nb = c->t.nb;
    r.nv = c->t.nv;
    r.nc = c->t.nc;
    return r;
}

// the direct kernel on the context's own tasks (its system as a kernel parameter)
static int direct_single(bse_ctx* c, int p32, const PairTask* tasks, int64_t n, void* X) {
    DirectInst di;
    di.S = c->S;
    di.coef = p32 ? c->coef32.p : (const void*)c->S.coef;
    di.w = p32 ? c->w32.p : (const void*)c->S.w;
    return launch_direct(di, p32, tasks, n, X, c->stream);
}

extern "C" {

const char* bse_last_error(void) { return bse::last_error(); }

int bse_create(bse_ctx** out, const bse_system* sys, void* stream) {
    clear_error();
    if (!out || !sys) return fail(BSE_EINVAL, "null argument");
    *out = nullptr;
    bse_ctx* c = new (std::nothrow) bse_ctx();
    if (!c) return fail(BSE_ENOMEM, "out of host memory");
    c->stream = (cudaStream_t)stream;
    AllocStream alloc_on_(c->stream);
    int r = keep_pool_memory();
    if (r == BSE_OK) r = create_impl(c, sys);
    if (r != BSE_OK) {
        cudaStreamSynchronize(c->stream);
        free_ctx(c);
        return r;
    }
    *out = c;
    return BSE_OK;
}

int bse_destroy(bse_ctx* ctx) {
    if (!ctx) return BSE_OK;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
    return BSE_OK;
}

int bse_tables(const bse_ctx* c, bse_tables_view* v) {
    clear_error();
    if (!c || !v) return fail(BSE_EINVAL, "null argument");
    const Tables& t = c->t;
    v->n_ops = t.nops;
    v->nk = t.nk;
    v->n_stars = (int32_t)t.star_rep.size();
    v->n_irreps = t.n_irreps;
    v->n_orbits = (int32_t)t.orbit_star.size();
    v->n_product = t.N;
    v->rotk = t.rotk.data();
    v->star_of_k = t.star_of.data();
    v->star_rep = t.star_rep.data();
    v->s_k = t.s_k.data();
    v->class_of_op = t.class_of.data();
    v->chi = t.chi.data();
    v->irrep_dim = t.irrep_dim.data();
    v->bright = t.bright.data();
    v->block_dim = c->block_dim.data();
    v->orbit_of = t.orbit_of.data();
    v->fold = t.fold.data();
    v->npw_max = (int32_t)(c->gk.size() / (3 * (size_t)t.nk));
    v->ng_max = (int32_t)(c->gq.size() / (3 * (size_t)t.nk));
    v->npw = c->npw.data();
    v->gk = c->gk.data();
    v->ng = c->ng.data();
    v->gq = c->gq.data();
    BSE_TRY(wdiv_host(c));
    v->w_div = c->w_div;
    for (int mu = 0; mu < t.n_irreps; ++mu) BSE_TRY(ensure_pmat(c, mu));
    v->partner_dim = c->partner_dim.data();
    return BSE_OK;
}

int bse_pairdens(bse_ctx* c, const int32_t* k, const int32_t* kp, int64_t npairs, int32_t bands, int32_t prec,
                 void* out) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || (npairs > 0 && (!k || !kp || !out))) return fail(BSE_EINVAL, "null argument");
    if (bands < 0 || bands > 2) return fail(BSE_EINVAL, "bands must be CC, VV or CV");
    if (prec != BSE_FP64 && prec != BSE_FP32 && prec != BSE_BF16_SPLIT && prec != BSE_FP16_SPLIT)
        return fail(BSE_EINVAL, "unknown precision %d", prec);
    if (npairs < 0 || npairs > (1ll << 31) - 1) return fail(BSE_EINVAL, "npairs out of range");
    if (npairs == 0) return BSE_OK;
    std::vector<int32_t> both((size_t)2 * npairs);
    for (int64_t i = 0; i < npairs; ++i) {
        if (k[i] < 0 || k[i] >= c->t.nk || kp[i] < 0 || kp[i] >= c->t.nk)
            return fail(BSE_EINVAL, "k index out of range at pair %lld", (long long)i);
        both[i] = k[i];
        both[npairs + i] = kp[i];
    }
    BSE_TRY(upload(c->pairs, both.data(), both.size(), c->stream));
    const int* d = (const int*)c->pairs.p;
    if (prec == BSE_FP64) return launch_pairdens(c->S, d, d + npairs, npairs, bands, 0, (double2*)out, c->stream);
    BSE_TRY(ensure_narrow(c));
    return launch_pairdens32(c->S, (const float2*)c->coef32.p, d, d + npairs, npairs, bands, (float2*)out,
                             c->stream);
}

int bse_build_full(bse_ctx* c, uint32_t terms, void* h, int64_t ld) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !h) return fail(BSE_EINVAL, "null argument");
    const Tables& t = c->t;
    if (ld < t.N || ld > (1ll << 31) - 1) return fail(BSE_EINVAL, "ld must be in [N, 2^31)");
    std::vector<PairTask> tasks;
    tasks.reserve((size_t)t.nk * (t.nk + 1) / 2);
    for (int k = 0; k < t.nk; ++k)
        for (int kp = k; kp < t.nk; ++kp) {
            PairTask p;
            p.k = k;
            p.kp = kp;
            p.row0 = k * t.B;
            p.col0 = kp * t.B;
            p.xoff = 0;
            p.ld = (int32_t)ld;
            p.flags = kp > k ? 1 : 0;
            tasks.push_back(p);
        }
    if (terms & BSE_TERM_DIRECT) {
        BSE_TRY(upload(c->tasks, tasks.data(), tasks.size(), c->stream));
        BSE_TRY(direct_single(c, 0, (const PairTask*)c->tasks.p, (int64_t)tasks.size(), h));
    } else {
        BSE_CUDA(cudaMemset2DAsync(h, sizeof(double2) * ld, 0, sizeof(double2) * t.N, t.N, c->stream));
    }
    if (terms & BSE_TERM_DIAG)
        BSE_TRY(launch_diag_full((const double*)c->de.p, t.N, (const double*)c->wdivDev.p, (double2*)h, ld, c->stream));
    if (terms & BSE_TERM_EXCHANGE) {
        BSE_TRY(ensure_exchange_vectors(c));
        BSE_TRY(launch_exchange_full((const double2*)c->P.p, (const double*)c->vbar.p, c->ng0, t.N,
                                     c->spin * c->S.inv_vol, (double2*)h, ld, c->stream));
    }
    return BSE_OK;
}

// The tensor-core kernel takes groups of up to kg pairs with the same
// q = k - k' (they share W(q)): the tasks sorted by q (stable) and their groups.
static void tc_group_tasks(const Tables& t, const std::vector<PairTask>& in, int kg, std::vector<PairTask>& sorted,
                           std::vector<TcGroup>& groups, int inst = 0, int32_t task_base = 0) {
    std::vector<int> qof(in.size());
    for (size_t i = 0; i < in.size(); ++i) {
        int iq[3];
        for (int a = 0; a < 3; ++a) iq[a] = (t.kidx[3 * in[i].k + a] - t.kidx[3 * in[i].kp + a] + t.n[a]) % t.n[a];
        qof[i] = (iq[0] * t.n[1] + iq[1]) * t.n[2] + iq[2];
    }
    std::vector<size_t> order(in.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return qof[a] < qof[b]; });
    sorted.resize(in.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = in[order[i]];
    groups.clear();
    for (size_t i = 0; i < order.size();) {
        TcGroup gp;
        gp.first = task_base + (int32_t)i;
        gp.q = qof[order[i]];
        gp.count = 0;
        gp.inst = inst;
        while (i < order.size() && qof[order[i]] == gp.q && gp.count < kg) {
            ++gp.count;
            ++i;
        }
        groups.push_back(gp);
    }
}

// U^dagger H U for an orbit-sparse basis U (an irrep block or a partner block)
// One build of several blocks (whole irrep blocks or partner blocks): the
// direct term of every star pair runs once per batch and each target projects
// the same X tiles with its own basis (Eqs. transformationU, Hblock).
// device copies of the tables the enumeration of rotated k pairs reads
static int ensure_rot_tables(bse_ctx* c) {
    if (c->rtab_ready) return BSE_OK;
    const Tables& t = c->t;
    std::vector<int> inv(t.nops, -1);
    for (int a = 0; a < t.nops; ++a)
        for (int b = 0; b < t.nops; ++b)
            if (t.mult[(size_t)a * t.nops + b] == t.identity) inv[a] = b;
    std::vector<int> all(t.mult.begin(), t.mult.end());
    const size_t o_inv = all.size();
    all.insert(all.end(), inv.begin(), inv.end());
    const size_t o_sk = all.size();
    all.insert(all.end(), t.s_k.begin(), t.s_k.end());
    const size_t o_pos = all.size();
    all.insert(all.end(), t.pos_in_star.begin(), t.pos_in_star.end());
    const size_t o_off = all.size();
    int run = 0;
    for (const auto& st : t.stars) {
        all.push_back(run);
        run += (int)st.size();
    }
    all.push_back(run);
    const size_t o_k = all.size();
    for (const auto& st : t.stars) all.insert(all.end(), st.begin(), st.end());
    BSE_TRY(upload(c->rtab_buf, all.data(), all.size(), c->stream));
    const int* b = (const int*)c->rtab_buf.p;
    c->rtab.rotk = (const int*)c->rotk.p;
    c->rtab.mult = b;
    c->rtab.inv = b + o_inv;
    c->rtab.s_k = b + o_sk;
    c->rtab.pos_in_star = b + o_pos;
    c->rtab.star_off = b + o_off;
    c->rtab.star_k = b + o_k;
    c->rtab.nops = t.nops;
    c->rtab.nk = t.nk;
    c->rtab.B = t.B;
    BSE_CUDA(cudaStreamSynchronize(c->stream));   // the host vector goes out of scope
    c->rtab_ready = true;
    return BSE_OK;
}

// ---------------------------------------------------------------------------
// Autotuning of the tensor-core direct term: the pairs per CTA (kg, the k pairs
// sharing one W(q) in MMA1) of a class of systems with the same shapes.  Each
// candidate the shared memory and the 256 TMEM columns allow is timed once on
// the class's own tasks (a persistent launch, CUDA events on the stream) and the
// fastest is kept for the process.
// ---------------------------------------------------------------------------
namespace {
struct TcClassKey {
    int fp16, nv, nc, ngp, npw, ng;
    bool operator<(const TcClassKey& o) const {
        return std::tie(fp16, nv, nc, ngp, npw, ng) < std::tie(o.fp16, o.nv, o.nc, o.ngp, o.npw, o.ng);
    }
};
struct TcChoice {
    int kg = 1;
    float ms[3] = {-1.f, -1.f, -1.f};   // measured launch times for kg = 1, 2, 4 (-1: not a candidate)
};
std::mutex g_tune_mu;
std::map<TcClassKey, TcChoice> g_tc_tuned;

TcClassKey tc_key(const DevSys& s, int fp16, int ngp) { return {fp16, s.nv, s.nc, ngp, s.npw_max, s.ng_max}; }

std::string tc_choice_json(const TcClassKey& k, const TcChoice& c, int instances) {
    char buf[320];
    std::snprintf(buf, sizeof buf,
                  "{\"class\": \"nv=%d nc=%d NGp=%d npw_max=%d ng_max=%d %s\", \"instances\": %d, "
                  "\"pairs_per_cta\": %d, \"threads_per_cta\": 256, \"ms\": {\"1\": %.4g, \"2\": %.4g, \"4\": %.4g}}",
                  k.nv, k.nc, k.ngp, k.npw, k.ng, k.fp16 ? "fp16" : "bf16", instances, c.kg, c.ms[0], c.ms[1],
                  c.ms[2]);
    return buf;
}
}  // namespace

// time the persistent tensor-core kernel on one system's tasks (xoff inside X) for each admissible kg
static int tune_tc(bse_ctx* c, int fp16, int ngp, const std::vector<PairTask>& tasks, void* X, int* status,
                   TcChoice& out) {
    out = TcChoice();
    if (tasks.empty()) return BSE_OK;
    DevBuf dt, dg, di, dq;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = BSE_OK;
    float best = -1.f;
    const int kgs[3] = {1, 2, 4};
    do {
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = fail(BSE_ECUDA, "autotuner events");
            break;
        }
        if ((rc = ensure(dq, sizeof(unsigned long long))) != BSE_OK) break;
        for (int j = 0; j < 3 && rc == BSE_OK; ++j) {
            const int kg = kgs[j];
            const size_t sm = tc_smem(c->S, ngp, kg);
            if (sm == 0) continue;
            TcInst ti{};
            ti.S = c->S;
            ti.coef = (const float2*)c->coef32.p;
            ti.wemb = c->wemb.p;
            ti.wexp = (const int*)c->wexp.p;
            ti.ngp = ngp;
            ti.kg = kg;
            std::vector<PairTask> sorted;
            std::vector<TcGroup> groups;
            tc_group_tasks(c->t, tasks, kg, sorted, groups);
            if ((rc = upload(dt, sorted.data(), sorted.size(), c->stream)) != BSE_OK) break;
            if ((rc = upload(dg, groups.data(), groups.size(), c->stream)) != BSE_OK) break;
            if ((rc = upload(di, &ti, 1, c->stream)) != BSE_OK) break;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && rc == BSE_OK; ++rep) {   // the first run warms up
                if (cudaMemsetAsync(dq.p, 0, sizeof(unsigned long long), c->stream) != cudaSuccess ||
                    cudaEventRecord(e0, c->stream) != cudaSuccess) {
                    rc = fail(BSE_ECUDA, "autotuner launch");
                    break;
                }
                rc = launch_direct_tc((const TcInst*)di.p, fp16, sm, (const PairTask*)dt.p, (const TcGroup*)dg.p,
                                      (int64_t)groups.size(), (unsigned long long*)dq.p, X, status, c->stream,
                                      c->wait_polls);
                if (rc == BSE_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess ||
                                     cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    rc = fail(BSE_ECUDA, "autotuner timing");
            }
            if (rc != BSE_OK) break;
            out.ms[j] = ms;
            if (best < 0.f || ms < best) {
                best = ms;
                out.kg = kg;
            }
        }
    } while (0);
    release(dt);
    release(dg);
    release(di);
    release(dq);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

// the tuned kg of a system's class (tuned on these tasks on first use)
static int tc_pairs_per_cta(bse_ctx* c, int fp16, int ngp, const std::vector<PairTask>& tasks, void* X, int* status,
                            int* kg) {
    const TcClassKey key = tc_key(c->S, fp16, ngp);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tc_tuned.find(key);
        if (it != g_tc_tuned.end()) {
            *kg = it->second.kg;
            return BSE_OK;
        }
    }
    TcChoice ch;
    BSE_TRY(tune_tc(c, fp16, ngp, tasks, X, status, ch));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tc_tuned[key] = ch;
    *kg = ch.kg;
    return BSE_OK;
}

static int build_multi(bse_ctx* c, const std::vector<IrrepDev*>& tg, int32_t prec, uint32_t terms,
                       void* const* h, const int64_t* ld) {
    const int tcp = prec == BSE_BF16_SPLIT || prec == BSE_FP16_SPLIT;
    const int fp16 = prec == BSE_FP16_SPLIT;
    const int p32 = prec == BSE_FP32 || tcp;   // the tile arena is FP32 for all three
    int ngp = 0, tc_group = 1;
    if (tcp && (terms & BSE_TERM_DIRECT)) {
        size_t sm = 0;
        BSE_TRY(tc_supported(c->S, ngp, sm, &tc_group));
    }
    const Tables& t = c->t;
    const size_t nt = tg.size();
    std::vector<const Basis*> bases;
    std::vector<DevBasis> db;
    std::vector<int64_t> pmu_off(nt + 1, 0);
    int64_t total = 0;
    for (size_t i = 0; i < nt; ++i) {
        if (ld[i] < tg[i]->host.dim) return fail(BSE_EINVAL, "target %zu: ld < block dimension", i);
        if (tg[i]->host.dim > 0 && !h[i]) return fail(BSE_EINVAL, "target %zu: null output", i);
        bases.push_back(&tg[i]->host);
        db.push_back(dev_basis_of(c, *tg[i]));
        pmu_off[i + 1] = pmu_off[i] + tg[i]->host.dim * c->ng0;
        total += tg[i]->host.dim;
    }
    if (total == 0) return BSE_OK;
    if (c->timing) c->stats.ms_exchange = 0.f;
    if (terms & BSE_TERM_EXCHANGE) {
        BSE_TRY(ensure_exchange_vectors(c));
        BSE_TRY(ensure(c->Pmu, sizeof(double2) * (size_t)pmu_off[nt]));
        if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[3], c->stream));
        for (size_t i = 0; i < nt; ++i)
            if (db[i].dim > 0)
                BSE_TRY(launch_exchange_project(db[i], (const double2*)c->P.p, c->ng0,
                                                (double2*)c->Pmu.p + pmu_off[i], c->stream));
        if (p32) {   // the mixed builds project the exchange in double-float: v^1/2-scaled copies
            BSE_TRY(ensure(c->Pt, sizeof(float4) * (size_t)pmu_off[nt]));
            BSE_TRY(launch_exchange_df((const double2*)c->Pmu.p, (const double*)c->vbar.p, pmu_off[nt] / c->ng0,
                                       c->ng0, (float4*)c->Pt.p, c->stream));
        }
        if (c->timing) {
            BSE_CUDA(cudaEventRecord(c->ev[4], c->stream));
            BSE_CUDA(cudaEventSynchronize(c->ev[4]));
            BSE_CUDA(cudaEventElapsedTime(&c->stats.ms_exchange, c->ev[3], c->ev[4]));
        }
    }
    if (p32 && (terms & BSE_TERM_DIRECT)) BSE_TRY(ensure_narrow(c));
    const bool dev_rots = c->seeds && (terms & BSE_TERM_DIRECT);   // rotated pairs enumerated on the device
    if (tcp && (terms & BSE_TERM_DIRECT)) BSE_TRY(ensure_wemb(c, ngp, fp16));
    if ((tcp && (terms & BSE_TERM_DIRECT)) || dev_rots) {
        BSE_TRY(ensure(c->status, sizeof(int)));
        BSE_CUDA(cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream));
    }
    if (dev_rots) BSE_TRY(ensure_rot_tables(c));
    const size_t xel = p32 ? sizeof(float2) : sizeof(double2);
    std::vector<Batch> batches;
    BSE_TRY(plan_batches(t, bases, arena_budget(), batches, dev_rots, false));
    if (c->timing) {
        c->stats.ms_direct = c->stats.ms_project = c->stats.ms_rotate = 0.f;
        c->stats.direct_launches = 0;
    }
    for (const Batch& bt : batches) {
        size_t ymax = 0;
        for (size_t y : bt.ybytes) ymax = std::max(ymax, y);
        BSE_TRY(ensure(c->arenaX, bt.xbytes / sizeof(double2) * xel));
        BSE_TRY(ensure(c->arenaY, ymax));
        std::vector<TcGroup> groups;
        size_t tc_sm = 0;
        if (tcp && (terms & BSE_TERM_DIRECT)) {
            // pairs per CTA tuned for this class of systems (on this batch's tasks, first use only)
            BSE_TRY(tc_pairs_per_cta(c, fp16, ngp, bt.tasks, c->arenaX.p, (int*)c->status.p, &tc_group));
            tc_sm = tc_smem(c->S, ngp, tc_group);
            std::vector<PairTask> sorted;
            tc_group_tasks(t, bt.tasks, tc_group, sorted, groups);
            BSE_TRY(upload(c->tasks, sorted.data(), sorted.size(), c->stream));
            BSE_TRY(upload(c->groups, groups.data(), groups.size(), c->stream));
            TcInst ti{};
            ti.S = c->S;
            ti.coef = (const float2*)c->coef32.p;
            ti.wemb = c->wemb.p;
            ti.wexp = (const int*)c->wexp.p;
            ti.ngp = ngp;
            ti.kg = tc_group;
            BSE_TRY(upload(c->tcinst, &ti, 1, c->stream));
            BSE_TRY(ensure(c->tcq, sizeof(unsigned long long)));
            c->stats.tc_pairs_per_cta = tc_group;
        } else {
            BSE_TRY(upload(c->tasks, bt.tasks.data(), bt.tasks.size(), c->stream));
        }
        BSE_TRY(upload(c->tiles, bt.tiles.data(), bt.tiles.size(), c->stream));
        if ((terms & BSE_TERM_DIRECT) && bt.nrots > 0) {
            // before any launch of the batch: a pageable copy waits for the stream to drain
            BSE_TRY(upload(c->rtiles, bt.rtiles.data(), bt.rtiles.size(), c->stream));
            BSE_TRY(upload(c->rmeta, bt.rmeta.data(), bt.rmeta.size(), c->stream));
            BSE_TRY(ensure(c->rots, sizeof(RotTask) * (size_t)bt.nrots));
        }
        if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[0], c->stream));
        if ((terms & BSE_TERM_DIRECT) && tcp) {
            BSE_CUDA(cudaMemsetAsync(c->tcq.p, 0, sizeof(unsigned long long), c->stream));
            BSE_TRY(launch_direct_tc((const TcInst*)c->tcinst.p, fp16, tc_sm, (const PairTask*)c->tasks.p,
                                     (const TcGroup*)c->groups.p, (int64_t)groups.size(),
                                     (unsigned long long*)c->tcq.p, c->arenaX.p, (int*)c->status.p, c->stream,
                                     c->wait_polls));
        } else if (terms & BSE_TERM_DIRECT) {
            BSE_TRY(direct_single(c, p32, (const PairTask*)c->tasks.p, (int64_t)bt.tasks.size(), c->arenaX.p));
        } else {
            BSE_CUDA(cudaMemsetAsync(c->arenaX.p, 0, bt.xbytes / sizeof(double2) * xel, c->stream));
        }
        if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[8], c->stream));
        if ((terms & BSE_TERM_DIRECT) && bt.nrots > 0) {   // the other pairs from their seeds (Eq. Wtrafo)
            const int* jr = (const int*)c->rmeta.p;
            const size_t nm = bt.rmeta.size() / 3;
            BSE_TRY(launch_rot_tasks(c->rtab, (const RotTile*)c->rtiles.p, (int)bt.rtiles.size(), bt.npairs, jr,
                                     jr + nm, jr + 2 * nm, (RotTask*)c->rots.p, (int*)c->status.p, c->stream));
            BSE_TRY(launch_rotate(rot_sys(c, p32), p32, (const RotTask*)c->rots.p, bt.nrots, c->arenaX.p,
                                  c->stream));
        }
        if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[1], c->stream));
        for (size_t i = 0; i < nt; ++i) {
            const int n = bt.tile_off[i + 1] - bt.tile_off[i];
            if (n == 0) continue;
            const TileTask* tl = (const TileTask*)c->tiles.p + bt.tile_off[i];
            // the mixed builds keep Y in double-float between the two stages (same 16 bytes per element)
            BSE_TRY(launch_project_right(db[i], tl, n, p32, c->arenaX.p, (double2*)c->arenaY.p, bt.max_rows[i],
                                         bt.max_cb[i], c->stream, p32));
            BSE_TRY(launch_project_left(db[i], tl, n, (const double2*)c->arenaY.p,
                                        (terms & BSE_TERM_EXCHANGE) ? (const double2*)c->Pmu.p + pmu_off[i] : nullptr,
                                        (const double*)c->vbar.p, c->ng0, c->spin * c->S.inv_vol,
                                        (terms & BSE_TERM_DIAG) ? (const double*)c->de.p : nullptr, (const double*)c->wdivDev.p,
                                        (double2*)h[i], ld[i], bt.max_ca[i], bt.max_cb[i], c->stream, p32,
                                        (terms & BSE_TERM_EXCHANGE) && p32 ? (const float4*)c->Pt.p + pmu_off[i] : nullptr));
        }
        if (c->timing) {
            BSE_CUDA(cudaEventRecord(c->ev[2], c->stream));
            BSE_CUDA(cudaEventSynchronize(c->ev[2]));
            float a = 0.f, b = 0.f, r = 0.f;
            BSE_CUDA(cudaEventElapsedTime(&a, c->ev[0], c->ev[1]));
            BSE_CUDA(cudaEventElapsedTime(&b, c->ev[1], c->ev[2]));
            BSE_CUDA(cudaEventElapsedTime(&r, c->ev[8], c->ev[1]));
            c->stats.ms_rotate += r;
            c->stats.ms_direct += a;
            c->stats.ms_project += b;
            c->stats.direct_launches += 1;
        }
    }
    if ((tcp && (terms & BSE_TERM_DIRECT)) || dev_rots) {
        int st = 0;
        BSE_CUDA(cudaMemcpyAsync(&st, c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        BSE_CUDA(cudaStreamSynchronize(c->stream));
        if (st & 2) return fail(BSE_ESYMM, "the seed of a rotated k pair was not found");
        if (st & 1) return fail(BSE_ETIMEOUT, "a bounded wait of the tensor-core direct kernel gave up");
    }
    return BSE_OK;
}

static int build_generic(bse_ctx* c, IrrepDev& bd, int32_t prec, uint32_t terms, void* h, int64_t ld) {
    std::vector<IrrepDev*> tg{&bd};
    return build_multi(c, tg, prec, terms, &h, &ld);
}

int bse_build_block(bse_ctx* c, int32_t mu, int32_t prec, uint32_t terms, void* h, int64_t ld) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !h) return fail(BSE_EINVAL, "null argument");
    if (prec != BSE_FP64 && prec != BSE_FP32 && prec != BSE_BF16_SPLIT && prec != BSE_FP16_SPLIT)
        return fail(BSE_EUNSUPPORTED, "precision %d is not implemented", prec);
    if (mu == BSE_IRREP_ALL) {   // every block, packed one after another in irrep order
        std::vector<IrrepDev*> tg;
        std::vector<void*> hs;
        std::vector<int64_t> lds;
        size_t off = 0;
        for (int m = 0; m < c->t.n_irreps; ++m) {
            BSE_TRY(ensure_basis(c, m));
            const int64_t d = c->irr[m].host.dim;
            tg.push_back(&c->irr[m]);
            hs.push_back(d > 0 ? (void*)((double2*)h + off) : nullptr);
            lds.push_back(std::max<int64_t>(d, 1));
            off += (size_t)d * d;
        }
        return build_multi(c, tg, prec, terms, hs.data(), lds.data());
    }
    BSE_TRY(ensure_basis(c, mu));
    return build_generic(c, c->irr[mu], prec, terms, h, ld);
}

int bse_build_partner_block(bse_ctx* c, int32_t mu, int32_t prec, uint32_t terms, void* h, int64_t ld) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !h) return fail(BSE_EINVAL, "null argument");
    if (prec != BSE_FP64 && prec != BSE_FP32 && prec != BSE_BF16_SPLIT && prec != BSE_FP16_SPLIT)
        return fail(BSE_EUNSUPPORTED, "precision %d is not implemented", prec);
    BSE_TRY(ensure_partner(c, mu));
    return build_generic(c, c->partner[mu].part[0], prec, terms, h, ld);
}

int bse_build_blocks(bse_ctx* c, int32_t n, const int32_t* irrep, const int32_t* partner, int32_t prec,
                     uint32_t terms, void* const* h, const int64_t* ld) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || n < 0 || (n > 0 && (!irrep || !h || !ld))) return fail(BSE_EINVAL, "null argument");
    if (prec != BSE_FP64 && prec != BSE_FP32 && prec != BSE_BF16_SPLIT && prec != BSE_FP16_SPLIT)
        return fail(BSE_EUNSUPPORTED, "precision %d is not implemented", prec);
    std::vector<IrrepDev*> tg;
    for (int32_t i = 0; i < n; ++i) {
        if (partner && partner[i]) {
            BSE_TRY(ensure_partner(c, irrep[i]));
            tg.push_back(&c->partner[irrep[i]].part[0]);
        } else {
            BSE_TRY(ensure_basis(c, irrep[i]));
            tg.push_back(&c->irr[irrep[i]]);
        }
    }
    if (n == 0) return BSE_OK;
    return build_multi(c, tg, prec, terms, h, ld);
}

// ---------------------------------------------------------------------------
// batched build: one block per context, the direct terms of all contexts in
// one launch, the projections per context, captured once as a CUDA graph
// ---------------------------------------------------------------------------
struct bse_batch {
    std::vector<bse_ctx*> ctx;
    std::vector<IrrepDev*> tg;
    std::vector<void*> h;
    std::vector<int64_t> ld;
    cudaStream_t stream = nullptr;
    DevBuf insts, tasks, tiles, arenaX, pmu, rsys, rots;
    int64_t nrots = 0;
    int bmax = 0;
    // split precisions: one persistent tensor-core launch over the q-sorted groups of all instances
    std::vector<int> tc_ngp;       // per instance
    int tcp = 0, fp16 = 0;
    int64_t tc_ngroups = 0;
    size_t tc_smem_max = 0;
    DevBuf tctasks, tcgroups, status, tcinsts, queue;
    // FP32 / FP64: one persistent launch of the direct kernel over the tasks of all instances
    int64_t ntasks = 0;
    DevSys smax{};
    int direct_threads = 256;
    std::string tuning;           // the autotuner's choices (JSON)
    static constexpr int kBranches = 4;   // concurrent projection branches of the graph
    DevBuf arenaY[kBranches];
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;          // kernel nodes in the graph
};

static void free_batch(bse_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (DevBuf* d : {&b->insts, &b->tasks, &b->tiles, &b->arenaX, &b->pmu, &b->rsys, &b->rots, &b->tctasks,
                      &b->tcgroups, &b->status, &b->tcinsts, &b->queue})
        release(*d);
    for (auto& y : b->arenaY) release(y);
    delete b;
}

// the launches of one batched build, captured into the graph on stream st:
// the direct term (one persistent launch), then the exchange and the
// projections of the instances on kBranches concurrent branches (fork/join
// through events), each branch with its own Y arena
static int batch_launches(bse_batch* b, cudaStream_t st, cudaStream_t* br, cudaEvent_t* ev, int p32, uint32_t terms,
                          const std::vector<Batch>& plans, const std::vector<int64_t>& pmu_off,
                          const std::vector<int>& tile_off,
                          const std::vector<int>& order) {
    const int nb = bse_batch::kBranches;
    if ((terms & BSE_TERM_DIRECT) && b->tcp) {   // one persistent launch over every instance's groups
        BSE_CUDA(cudaMemsetAsync(b->status.p, 0, sizeof(int), st));
        BSE_CUDA(cudaMemsetAsync(b->queue.p, 0, sizeof(unsigned long long), st));
        BSE_TRY(launch_direct_tc((const TcInst*)b->tcinsts.p, b->fp16, b->tc_smem_max, (const PairTask*)b->tctasks.p,
                                 (const TcGroup*)b->tcgroups.p, b->tc_ngroups, (unsigned long long*)b->queue.p,
                                 b->arenaX.p, (int*)b->status.p, st, b->ctx[0]->wait_polls));
    }
    if (terms & BSE_TERM_DIRECT) {
        if (!b->tcp && b->ntasks > 0) {   // one persistent launch over every instance's tasks
            BSE_CUDA(cudaMemsetAsync(b->queue.p, 0, sizeof(unsigned long long), st));
            BSE_TRY(launch_direct_persistent((const DirectInst*)b->insts.p, b->smax, p32, (const PairTask*)b->tasks.p,
                                             b->ntasks, (unsigned long long*)b->queue.p, b->direct_threads, 0,
                                             b->arenaX.p, st));
        }
        if (b->nrots > 0)   // pairs rotated from their seeds (Eq. Wtrafo)
            BSE_TRY(launch_rotate_multi((const RotSys*)b->rsys.p, b->bmax, p32, (const RotTask*)b->rots.p, b->nrots,
                                        b->arenaX.p, st));
    } else {
        BSE_CUDA(cudaMemsetAsync(b->arenaX.p, 0, b->arenaX.n, st));
    }
    BSE_CUDA(cudaEventRecord(ev[0], st));
    for (int j = 0; j < nb; ++j) BSE_CUDA(cudaStreamWaitEvent(br[j], ev[0], 0));
    for (size_t q = 0; q < order.size(); ++q) {
        const int i = order[q];
        const int j = (int)(q % nb);
        bse_ctx* c = b->ctx[i];
        if (b->tg[i]->host.dim == 0) continue;
        DevBasis db = dev_basis_of(c, *b->tg[i]);
        if (terms & BSE_TERM_EXCHANGE)
            BSE_TRY(launch_exchange_project(db, (const double2*)c->P.p, c->ng0, (double2*)b->pmu.p + pmu_off[i], br[j]));
        const Batch& bt = plans[i];
        const int nt = (int)bt.tiles.size();
        if (nt == 0) continue;
        const TileTask* tl = (const TileTask*)b->tiles.p + tile_off[i];   // xoff already global in the arena
        BSE_TRY(launch_project_right(db, tl, nt, p32, b->arenaX.p, (double2*)b->arenaY[j].p, bt.max_rows[0],
                                     bt.max_cb[0], br[j]));
        BSE_TRY(launch_project_left(db, tl, nt, (const double2*)b->arenaY[j].p,
                                    (terms & BSE_TERM_EXCHANGE) ? (const double2*)b->pmu.p + pmu_off[i] : nullptr,
                                    (const double*)c->vbar.p, c->ng0, c->spin * c->S.inv_vol,
                                    (terms & BSE_TERM_DIAG) ? (const double*)c->de.p : nullptr, (const double*)c->wdivDev.p,
                                    (double2*)b->h[i], b->ld[i], bt.max_ca[0], bt.max_cb[0], br[j]));
    }
    for (int j = 0; j < nb; ++j) {
        BSE_CUDA(cudaEventRecord(ev[1 + j], br[j]));
        BSE_CUDA(cudaStreamWaitEvent(st, ev[1 + j], 0));
    }
    return BSE_OK;
}

static int batch_create_impl(bse_batch* b, int32_t n, const int32_t* irrep, const int32_t* partner, int32_t prec,
                             uint32_t terms, void* const* h, const int64_t* ld) {
    b->tcp = (prec == BSE_BF16_SPLIT || prec == BSE_FP16_SPLIT) && (terms & BSE_TERM_DIRECT);
    b->fp16 = prec == BSE_FP16_SPLIT;
    const int p32 = prec == BSE_FP32 || prec == BSE_BF16_SPLIT || prec == BSE_FP16_SPLIT;   // FP32 tile arena
    for (int32_t i = 0; i < n; ++i) {
        bse_ctx* c = b->ctx[i];
        if (partner && partner[i]) {
            BSE_TRY(ensure_partner(c, irrep[i]));
            b->tg.push_back(&c->partner[irrep[i]].part[0]);
        } else {
            BSE_TRY(ensure_basis(c, irrep[i]));
            b->tg.push_back(&c->irr[irrep[i]]);
        }
        if (ld[i] < b->tg[i]->host.dim) return fail(BSE_EINVAL, "instance %d: ld < block dimension", i);
        if (b->tg[i]->host.dim > 0 && !h[i]) return fail(BSE_EINVAL, "instance %d: null output", i);
        if (terms & BSE_TERM_EXCHANGE) BSE_TRY(ensure_exchange_vectors(c));
        if (p32 && (terms & BSE_TERM_DIRECT)) BSE_TRY(ensure_narrow(c));
        if (b->tcp) {
            int ngp = 0;
            size_t sm = 0;
            BSE_TRY(tc_supported(c->S, ngp, sm));
            BSE_TRY(ensure_wemb(c, ngp, b->fp16));
            b->tc_ngp.push_back(ngp);
        }
        b->h.push_back(h[i]);
        b->ld.push_back(ld[i]);
    }
    // one plan (one arena batch) per instance; tasks and tiles concatenated
    std::vector<Batch> plans(n);
    std::vector<int64_t> xbase(n + 1, 0), pmu_off(n + 1, 0);
    std::vector<int> tile_off(n + 1, 0);
    std::vector<TileTask> tiles;
    std::vector<DirectInst> insts(n);
    std::vector<RotSys> rsys(n);
    std::vector<RotTask> rots;
    std::vector<size_t> ysz(n, 0);
    for (int32_t i = 0; i < n; ++i) {
        bse_ctx* c = b->ctx[i];
        std::vector<Batch> bb;
        BSE_TRY(plan_batches(c->t, std::vector<const Basis*>{&b->tg[i]->host}, (size_t)1 << 62, bb,
                             c->seeds && (terms & BSE_TERM_DIRECT)));
        if (bb.size() > 1) return fail(BSE_EUNSUPPORTED, "instance %d: tiles do not fit one arena", i);
        if (!bb.empty()) plans[i] = std::move(bb[0]);
        else {
            plans[i].max_rows.assign(1, 0);
            plans[i].max_ca.assign(1, 0);
            plans[i].max_cb.assign(1, 0);
            plans[i].ybytes.assign(1, 0);
        }
        const int64_t xel_count = (int64_t)(plans[i].xbytes / sizeof(double2));
        xbase[i + 1] = xbase[i] + xel_count;
        tile_off[i] = (int)tiles.size();
        for (TileTask t : plans[i].tiles) {
            t.xoff += xbase[i];
            tiles.push_back(t);
        }
        tile_off[i + 1] = (int)tiles.size();
        ysz[i] = plans[i].ybytes.empty() ? (size_t)0 : plans[i].ybytes[0];
        pmu_off[i + 1] = pmu_off[i] + b->tg[i]->host.dim * c->ng0;
        insts[i].S = c->S;
        insts[i].coef = p32 ? c->coef32.p : (const void*)c->S.coef;
        insts[i].w = p32 ? c->w32.p : (const void*)c->S.w;
        rsys[i] = rot_sys(c, p32);
        b->bmax = std::max(b->bmax, c->t.nv * c->t.nc);
        for (RotTask r : plans[i].rots) {
            r.src += xbase[i];
            r.dst += xbase[i];
            r.dstm += xbase[i];
            r.flags |= i << 1;
            rots.push_back(r);
        }
    }
    b->nrots = (int64_t)rots.size();
    const size_t xel = p32 ? sizeof(float2) : sizeof(double2);
    BSE_TRY(ensure(b->arenaX, (size_t)xbase[n] * xel));
    BSE_TRY(ensure(b->queue, sizeof(unsigned long long)));
    BSE_TRY(ensure(b->status, sizeof(int)));
    // instances in decreasing order of their direct-term work per k pair, so that the work queue
    // of the persistent launch hands out the longest tasks first
    std::vector<int> bycost(n);
    for (int32_t i = 0; i < n; ++i) bycost[i] = i;
    auto pair_cost = [&](int i) {
        const DevSys& sy = b->ctx[i]->S;
        return (double)sy.ng_max * ((double)sy.nv * sy.nv * sy.ng_max + (double)sy.nc * sy.nc * sy.nv * sy.nv) +
               (double)sy.npw_max * sy.ng_max * (sy.nc * sy.nc + sy.nv * sy.nv);
    };
    std::stable_sort(bycost.begin(), bycost.end(), [&](int x, int y) { return pair_cost(x) > pair_cost(y); });
    std::string tune = "{";
    if (b->tcp && (terms & BSE_TERM_DIRECT)) {
        // pairs per CTA of each class of instances (tuned on the class's first instance), then one
        // group list over all instances for the persistent tensor-core launch
        std::vector<TcInst> tinst(n);
        std::vector<PairTask> tctasks;
        std::vector<TcGroup> tcgroups;
        std::map<TcClassKey, int> class_count;
        for (int q = 0; q < n; ++q) {
            const int i = bycost[q];
            bse_ctx* c = b->ctx[i];
            std::vector<PairTask> in(plans[i].tasks);
            for (PairTask& t : in) t.xoff += xbase[i];
            int kg = 1;
            BSE_TRY(tc_pairs_per_cta(c, b->fp16, b->tc_ngp[i], in, b->arenaX.p, (int*)b->status.p, &kg));
            class_count[tc_key(c->S, b->fp16, b->tc_ngp[i])] += 1;
            TcInst& ti = tinst[i];
            ti.S = c->S;
            ti.coef = (const float2*)c->coef32.p;
            ti.wemb = c->wemb.p;
            ti.wexp = (const int*)c->wexp.p;
            ti.ngp = b->tc_ngp[i];
            ti.kg = kg;
            b->tc_smem_max = std::max(b->tc_smem_max, tc_smem(c->S, ti.ngp, kg));
            std::vector<PairTask> sorted;
            std::vector<TcGroup> gr;
            tc_group_tasks(c->t, in, kg, sorted, gr, i, (int32_t)tctasks.size());
            tctasks.insert(tctasks.end(), sorted.begin(), sorted.end());
            tcgroups.insert(tcgroups.end(), gr.begin(), gr.end());
        }
        b->tc_ngroups = (int64_t)tcgroups.size();
        BSE_TRY(upload(b->tctasks, tctasks.data(), tctasks.size(), b->stream));
        BSE_TRY(upload(b->tcgroups, tcgroups.data(), tcgroups.size(), b->stream));
        BSE_TRY(upload(b->tcinsts, tinst.data(), tinst.size(), b->stream));
        tune += "\"direct_kernel\": \"direct_tc_kernel (persistent, one launch)\", \"classes\": [";
        bool first = true;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto& kv : class_count) {
            tune += (first ? "" : ", ") + tc_choice_json(kv.first, g_tc_tuned[kv.first], kv.second);
            first = false;
        }
        tune += "]";
    } else if (terms & BSE_TERM_DIRECT) {
        // FP32 / FP64: every instance's tasks in one list for the persistent direct kernel
        std::vector<PairTask> tasks_all;
        for (int q = 0; q < n; ++q) {
            const int i = bycost[q];
            const DevSys& sy = b->ctx[i]->S;
            if (q == 0) b->smax = sy;
            b->smax.nb = std::max(b->smax.nb, sy.nb);
            b->smax.nv = std::max(b->smax.nv, sy.nv);
            b->smax.nc = std::max(b->smax.nc, sy.nc);
            b->smax.npw_max = std::max(b->smax.npw_max, sy.npw_max);
            b->smax.ng_max = std::max(b->smax.ng_max, sy.ng_max);
            for (PairTask t : plans[i].tasks) {
                t.xoff += xbase[i];
                t.flags |= i << 1;
                tasks_all.push_back(t);
            }
        }
        b->ntasks = (int64_t)tasks_all.size();
        BSE_TRY(upload(b->tasks, tasks_all.data(), tasks_all.size(), b->stream));
        BSE_TRY(upload(b->insts, insts.data(), insts.size(), b->stream));
        // threads per CTA of the persistent launch, timed on the batch's own tasks
        float ms[2] = {-1.f, -1.f};
        const int thr[2] = {128, 256};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        BSE_CUDA(cudaEventCreate(&e0));
        BSE_CUDA(cudaEventCreate(&e1));
        int rc = BSE_OK;
        for (int j = 0; j < 2 && rc == BSE_OK && b->ntasks > 0; ++j)
            for (int rep = 0; rep < 2 && rc == BSE_OK; ++rep) {
                if (cudaMemsetAsync(b->queue.p, 0, sizeof(unsigned long long), b->stream) != cudaSuccess ||
                    cudaEventRecord(e0, b->stream) != cudaSuccess) {
                    rc = fail(BSE_ECUDA, "autotuner launch");
                    break;
                }
                rc = launch_direct_persistent((const DirectInst*)b->insts.p, b->smax, p32, (const PairTask*)b->tasks.p,
                                              b->ntasks, (unsigned long long*)b->queue.p, thr[j], 0, b->arenaX.p,
                                              b->stream);
                if (rc == BSE_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess ||
                                     cudaEventSynchronize(e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&ms[j], e0, e1) != cudaSuccess))
                    rc = fail(BSE_ECUDA, "autotuner timing");
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        BSE_TRY(rc);
        b->direct_threads = (ms[0] >= 0.f && ms[0] < ms[1]) ? 128 : 256;
        char buf[256];
        std::snprintf(buf, sizeof buf,
                      "\"direct_kernel\": \"direct_persistent_kernel (one launch)\", \"threads_per_cta\": %d, "
                      "\"ms\": {\"128\": %.4g, \"256\": %.4g}", b->direct_threads, ms[0], ms[1]);
        tune += buf;
    }
    // the arena: one X arena holds every instance's tiles (its size in MB)
    {
        char buf[96];
        std::snprintf(buf, sizeof buf, "%s\"x_arena_mb\": %.1f}", tune.size() > 1 ? ", " : "",
                      (double)xbase[n] * xel / (1 << 20));
        tune += buf;
    }
    b->tuning = tune;
    // projection order: largest first, dealt round-robin to the branches
    std::vector<int> order(n);
    for (int32_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ysz[x] > ysz[y]; });
    size_t ybr[bse_batch::kBranches] = {0, 0, 0, 0};
    for (size_t q = 0; q < order.size(); ++q)
        ybr[q % bse_batch::kBranches] = std::max(ybr[q % bse_batch::kBranches], ysz[order[q]]);
    BSE_TRY(upload(b->tiles, tiles.data(), tiles.size(), b->stream));
    BSE_TRY(upload(b->rsys, rsys.data(), rsys.size(), b->stream));
    BSE_TRY(upload(b->rots, rots.data(), rots.size(), b->stream));
    for (int j = 0; j < bse_batch::kBranches; ++j) BSE_TRY(ensure(b->arenaY[j], ybr[j]));
    BSE_TRY(ensure(b->pmu, sizeof(double2) * (size_t)std::max<int64_t>(pmu_off[n], 1)));
    BSE_CUDA(cudaStreamSynchronize(b->stream));
    // capture on a stream of our own (the context's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the context's
    const int64_t l0 = launches_total();
    cudaStream_t cs = nullptr, br[bse_batch::kBranches] = {};
    cudaEvent_t ev[1 + bse_batch::kBranches] = {};
    auto cleanup = [&]() {
        for (auto& s : br)
            if (s) cudaStreamDestroy(s);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    };
    cudaError_t be = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (auto& s : br)
        if (be == cudaSuccess) be = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (auto& e : ev)
        if (be == cudaSuccess) be = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (be == cudaSuccess) be = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (be != cudaSuccess) {
        cleanup();
        return fail(BSE_ECUDA, "graph capture: %s", cudaGetErrorString(be));
    }
    const int rc = batch_launches(b, cs, br, ev, p32, terms, plans, pmu_off, tile_off, order);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    cleanup();
    if (rc != BSE_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return fail(BSE_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    b->graph = g;
    b->kernels = launches_total() - l0;
    BSE_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return BSE_OK;
}

int bse_batch_create(bse_batch** out, bse_ctx* const* ctxs, int32_t n, const int32_t* irrep, const int32_t* partner,
                     int32_t prec, uint32_t terms, void* const* h, const int64_t* ld) {
    clear_error();
    if (!out || !ctxs || n < 1 || !irrep || !h || !ld) return fail(BSE_EINVAL, "null argument");
    *out = nullptr;
    if (prec != BSE_FP64 && prec != BSE_FP32 && prec != BSE_BF16_SPLIT && prec != BSE_FP16_SPLIT)
        return fail(BSE_EUNSUPPORTED, "precision %d is not implemented", prec);
    for (int32_t i = 0; i < n; ++i) {
        if (!ctxs[i]) return fail(BSE_EINVAL, "null context %d", i);
        if (ctxs[i]->stream != ctxs[0]->stream) return fail(BSE_EINVAL, "contexts of a batch share one stream");
    }
    bse_batch* b = new (std::nothrow) bse_batch();
    if (!b) return fail(BSE_ENOMEM, "out of host memory");
    b->ctx.assign(ctxs, ctxs + n);
    b->stream = ctxs[0]->stream;
    AllocStream alloc_on_(b->stream);
    const int rc = batch_create_impl(b, n, irrep, partner, prec, terms, h, ld);
    if (rc != BSE_OK) {
        cudaStreamSynchronize(b->stream);
        free_batch(b);
        return rc;
    }
    *out = b;
    return BSE_OK;
}

int bse_batch_run(bse_batch* b) {
    clear_error();
    if (!b) return fail(BSE_EINVAL, "null batch");
    BSE_CUDA(cudaGraphLaunch(b->exec, b->stream));
    for (int64_t i = 0; i < b->kernels; ++i) note_launch();
    return BSE_OK;
}

int bse_batch_kernels(const bse_batch* b, int64_t* out) {
    clear_error();
    if (!b || !out) return fail(BSE_EINVAL, "null argument");
    *out = b->kernels;
    return BSE_OK;
}

int bse_batch_tuning(const bse_batch* b, char* buf, int64_t len) {
    clear_error();
    if (!b || !buf || len < 1) return fail(BSE_EINVAL, "null argument");
    const size_t m = std::min<size_t>(b->tuning.size(), (size_t)len - 1);
    std::memcpy(buf, b->tuning.data(), m);
    buf[m] = 0;
    return BSE_OK;
}

int bse_batch_destroy(bse_batch* b) {
    clear_error();
    if (!b) return BSE_OK;
    cudaStreamSynchronize(b->stream);
    int st = 0;
    if (b->tcp && b->status.p) cudaMemcpy(&st, b->status.p, sizeof(int), cudaMemcpyDeviceToHost);
    free_batch(b);
    if (st) return fail(BSE_ETIMEOUT, "a bounded wait of the tensor-core direct kernel gave up");
    return BSE_OK;
}

int bse_build_blocks_batched(bse_ctx* const* ctxs, int32_t n, const int32_t* irrep, const int32_t* partner,
                             int32_t prec, uint32_t terms, void* const* h, const int64_t* ld) {
    bse_batch* b = nullptr;
    BSE_TRY(bse_batch_create(&b, ctxs, n, irrep, partner, prec, terms, h, ld));
    const int rc = bse_batch_run(b);
    const int rd = bse_batch_destroy(b);   // waits; ETIMEOUT from a bounded wait of the run
    return rc != BSE_OK ? rc : rd;
}

int bse_block_dim(const bse_ctx* c, int32_t mu, int64_t* dim) {
    clear_error();
    if (!c || !dim) return fail(BSE_EINVAL, "null argument");
    if (mu == BSE_IRREP_ALL) {
        *dim = c->t.N;
        return BSE_OK;
    }
    if (mu < 0 || mu >= c->t.n_irreps) return fail(BSE_EINVAL, "irrep %d out of range [0, %d)", mu, c->t.n_irreps);
    *dim = c->block_dim[mu];
    return BSE_OK;
}

int bse_block_star_columns(bse_ctx* c, int32_t mu, int32_t partner, int64_t* out) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !out) return fail(BSE_EINVAL, "null argument");
    if (partner) BSE_TRY(ensure_partner(c, mu));
    else BSE_TRY(ensure_basis(c, mu));
    const Basis& bh = partner ? c->partner[mu].part[0].host : c->irr[mu].host;
    std::copy(bh.star_col.begin(), bh.star_col.end(), out);
    return BSE_OK;
}

int bse_block_basis(bse_ctx* c, int32_t mu, void* u, int64_t ld) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !u) return fail(BSE_EINVAL, "null argument");
    BSE_TRY(ensure_basis(c, mu));
    if (ld < c->t.N) return fail(BSE_EINVAL, "ld < N");
    const int64_t dim = c->irr[mu].host.dim;
    if (dim == 0) return BSE_OK;
    BSE_CUDA(cudaMemsetAsync(u, 0, sizeof(double2) * (size_t)ld * dim, c->stream));
    return launch_basis_dense(dev_basis(c, mu), (double2*)u, ld, c->stream);
}

int bse_dipoles(bse_ctx* c, void* b) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !b) return fail(BSE_EINVAL, "null argument");
    return launch_dipoles(c->S, (double2*)b, c->stream);
}

// eigensolution of U^dagger H U and the spectrum; the oscillator strength of
// each level sums |a^T (U_p^T B)|^2 over the given bases U_p (one for an
// irrep block, the d transfers for a partner block)
// Levels and strengths without eigenvectors (see bse_set_solver).  Returns
// BSE_OK when done; EUNSUPPORTED / ESOLVER when a condition of the path fails
// (the caller may fall back to the dense solver).
// The start direction of an eigenvector-free spectrum: the partner whose
// projection b_p = U_p^T B has the largest norm, and the total weight
// sum_p |b_p|^2 (0 for a dark irrep).  The partners' projections must be
// parallel (|G_pj|^2 = G_pp G_jj with G the Gram matrix), as they are for the
// partner blocks, so that one direction carries the whole measure.
static int start_direction(bse_ctx* c, int nparts, bool dark, int64_t dim, int* pmax_out, double* scale_out) {
    BSE_TRY(ensure(c->triSmall, 256));
    double2* gram = (double2*)c->triSmall.p;
    BSE_TRY(launch_gram((const double2*)c->Bmu.p, dim, nparts, gram, c->stream));
    double2 g[9];
    BSE_CUDA(cudaMemcpyAsync(g, gram, sizeof(g), cudaMemcpyDeviceToHost, c->stream));
    BSE_CUDA(cudaStreamSynchronize(c->stream));
    int pmax = 0;
    double scale = 0.0;
    for (int i = 0; i < nparts; ++i) {
        scale += g[i * 3 + i].x;
        if (g[i * 3 + i].x > g[pmax * 3 + pmax].x) pmax = i;
    }
    const double gpp = g[pmax * 3 + pmax].x;
    // an irrep outside the polar-vector representation has B_mu = 0 by symmetry: levels only
    if (dark) scale = 0.0;
    for (int j = 0; j < nparts && !dark; ++j) {
        const double gjj = g[j * 3 + j].x, a2 = g[pmax * 3 + j].x * g[pmax * 3 + j].x + g[pmax * 3 + j].y * g[pmax * 3 + j].y;
        if (gjj > 1e-20 * gpp && a2 < (1.0 - 1e-10) * gpp * gjj)
            return fail(BSE_EUNSUPPORTED, "the partners' dipole projections are not parallel");
    }
    *pmax_out = pmax;
    *scale_out = scale;
    return BSE_OK;
}

static int spectrum_tridiag(bse_ctx* c, int nparts, bool dark, int64_t dim, const void* h, int64_t ld,
                            double* omega_out, double* osc) {
    if (dim > tridiag_max_dim()) return fail(BSE_EUNSUPPORTED, "tridiagonal path: block dimension %lld > %d",
                                             (long long)dim, tridiag_max_dim());
    int pmax = 0;
    double scale = 0.0;
    BSE_TRY(start_direction(c, nparts, dark, dim, &pmax, &scale));
    double* wsum = (double*)((char*)c->triSmall.p + 160);
    int* err = (int*)((char*)c->triSmall.p + 176);
    BSE_TRY(ensure(c->eigA, sizeof(double2) * (size_t)dim * dim));
    BSE_CUDA(cudaMemcpy2DAsync(c->eigA.p, sizeof(double2) * dim, h, sizeof(double2) * ld, sizeof(double2) * dim, dim,
                               cudaMemcpyDeviceToDevice, c->stream));
    BSE_TRY(ensure(c->triScratch, tridiag_scratch_bytes(dim)));
    if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[3], c->stream));
    BSE_TRY(launch_tridiag_spectrum((double2*)c->eigA.p, dim, (const double2*)c->Bmu.p + (size_t)pmax * dim, scale,
                                    c->triScratch.p, omega_out, osc, wsum, err, c->stream,
                                    c->timing ? c->ev[6] : nullptr, c->timing ? c->ev[7] : nullptr, c->wait_polls,
                                    c->solver_mode == BSE_SOLVER_TRIDIAG_BLOCKED      ? 1
                                    : c->solver_mode == BSE_SOLVER_TRIDIAG_BLOCKED_DF ? 2
                                    : c->solver_mode == BSE_SOLVER_TRIDIAG_TWOSTAGE   ? 3
                                                                                      : 0,
                                    &c->stats.reduce_kind));
    if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[4], c->stream));
    struct {
        double s;
        int e;
    } chk{0.0, 0};
    BSE_CUDA(cudaMemcpyAsync(&chk.s, wsum, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BSE_CUDA(cudaMemcpyAsync(&chk.e, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BSE_CUDA(cudaStreamSynchronize(c->stream));
    if (chk.e) return fail(BSE_ETIMEOUT, "a grid barrier of the tridiagonal reduction gave up");
    if (scale > 0.0 && !(std::fabs(chk.s - 1.0) <= 1e-8))
        return fail(BSE_ESOLVER, "tridiagonal path: weights sum to %.17g instead of 1", chk.s);
    return BSE_OK;
}

static int spectrum_generic(bse_ctx* c, IrrepDev* parts, int nparts, int irrep_dim, bool dark, const void* h,
                            int64_t ld,
                            const double* omega, int64_t n_omega, double eta, double* omega_out, double* osc,
                            double* im_eps) {
    const int64_t dim = parts[0].host.dim;
    if (ld < dim) return fail(BSE_EINVAL, "ld < block dimension");
    if (dim == 0) {
        if (n_omega) BSE_CUDA(cudaMemsetAsync(im_eps, 0, sizeof(double) * n_omega, c->stream));
        return BSE_OK;
    }
    if (dim > (1ll << 31) - 1) return fail(BSE_EUNSUPPORTED, "block too large for the eigensolver");
    BSE_TRY(ensure_dipoles(c));
    BSE_TRY(ensure(c->Bmu, sizeof(double2) * (size_t)dim * nparts));
    for (int p = 0; p < nparts; ++p)
        BSE_TRY(launch_bmu(dev_basis_of(c, parts[p]), (const double2*)c->B.p, (double2*)c->Bmu.p + (size_t)p * dim,
                           c->stream));
    const double pref = 4.0 * M_PI * c->spin / c->t.nk;
    const bool forced_tri = c->solver_mode == BSE_SOLVER_TRIDIAG || c->solver_mode == BSE_SOLVER_TRIDIAG_BLOCKED ||
                            c->solver_mode == BSE_SOLVER_TRIDIAG_BLOCKED_DF || c->solver_mode == BSE_SOLVER_TRIDIAG_TWOSTAGE;
    const bool try_tri = forced_tri ||
                         (c->solver_mode == BSE_SOLVER_AUTO && (nparts > 1 || irrep_dim == 1 || dark) &&
                          dim <= tridiag_max_dim());
    if (try_tri) {
        const int rc = spectrum_tridiag(c, nparts, dark, dim, h, ld, omega_out, osc);
        if (rc == BSE_OK) {
            if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[4], c->stream));
            BSE_TRY(launch_spectrum(omega_out, osc, dim, omega, n_omega, eta, pref, im_eps, c->stream));
            if (c->timing) {
                BSE_CUDA(cudaEventRecord(c->ev[5], c->stream));
                BSE_CUDA(cudaEventSynchronize(c->ev[5]));
                BSE_CUDA(cudaEventElapsedTime(&c->stats.ms_eig, c->ev[3], c->ev[4]));
                BSE_CUDA(cudaEventElapsedTime(&c->stats.ms_spectrum, c->ev[4], c->ev[5]));
            }
            if (c->timing) BSE_CUDA(cudaEventElapsedTime(&c->stats.ms_reduce, c->ev[6], c->ev[7]));
            c->stats.solver = BSE_SOLVER_TRIDIAG;
            return BSE_OK;
        }
        if (forced_tri || rc == BSE_ETIMEOUT || rc == BSE_ECUDA)
            return rc;
        clear_error();
    }
    BSE_TRY(ensure(c->eigA, sizeof(double2) * (size_t)dim * dim));
    BSE_CUDA(cudaMemcpy2DAsync(c->eigA.p, sizeof(double2) * dim, h, sizeof(double2) * ld, sizeof(double2) * dim, dim,
                               cudaMemcpyDeviceToDevice, c->stream));
    if (!c->solver) {
        if (cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS) return fail(BSE_ESOLVER, "cusolverDnCreate failed");
    }
    if (cusolverDnSetStream(c->solver, c->stream) != CUSOLVER_STATUS_SUCCESS)
        return fail(BSE_ESOLVER, "cusolverDnSetStream failed");
    int lwork = 0;
    if (cusolverDnZheevd_bufferSize(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)dim,
                                    (const cuDoubleComplex*)c->eigA.p, (int)dim, omega_out,
                                    &lwork) != CUSOLVER_STATUS_SUCCESS)
        return fail(BSE_ESOLVER, "zheevd buffer size query failed");
    BSE_TRY(ensure(c->eigWork, sizeof(cuDoubleComplex) * (size_t)std::max(lwork, 1)));
    BSE_TRY(ensure(c->info, sizeof(int)));
    if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[3], c->stream));
    if (cusolverDnZheevd(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, (int)dim,
                         (cuDoubleComplex*)c->eigA.p, (int)dim, omega_out, (cuDoubleComplex*)c->eigWork.p, lwork,
                         (int*)c->info.p) != CUSOLVER_STATUS_SUCCESS)
        return fail(BSE_ESOLVER, "zheevd launch failed");
    if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[4], c->stream));
    BSE_TRY(launch_oscillators((const double2*)c->eigA.p, dim, dim, (const double2*)c->Bmu.p, nparts, osc,
                               c->stream));
    BSE_TRY(launch_spectrum(omega_out, osc, dim, omega, n_omega, eta, pref, im_eps, c->stream));
    if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[5], c->stream));
    int info = 0;
    BSE_CUDA(cudaMemcpyAsync(&info, c->info.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BSE_CUDA(cudaStreamSynchronize(c->stream));
    if (info != 0) return fail(BSE_ESOLVER, "zheevd info = %d", info);
    if (c->timing) {
        BSE_CUDA(cudaEventElapsedTime(&c->stats.ms_eig, c->ev[3], c->ev[4]));
        BSE_CUDA(cudaEventElapsedTime(&c->stats.ms_spectrum, c->ev[4], c->ev[5]));
    }
    c->stats.solver = BSE_SOLVER_DENSE;
    c->stats.ms_reduce = 0.f;
    return BSE_OK;
}

int bse_block_spectrum(bse_ctx* c, int32_t mu, const void* h, int64_t ld, const double* omega, int64_t n_omega,
                       double eta, double* omega_out, double* osc, double* im_eps) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !h || !omega_out || !osc || (n_omega > 0 && (!omega || !im_eps))) return fail(BSE_EINVAL, "null argument");
    if (!(eta > 0)) return fail(BSE_EINVAL, "eta must be positive");
    BSE_TRY(ensure_basis(c, mu));
    return spectrum_generic(c, &c->irr[mu], 1, c->t.irrep_dim[mu], !c->t.bright[mu], h, ld, omega, n_omega, eta,
                            omega_out, osc, im_eps);
}

int bse_partner_spectrum(bse_ctx* c, int32_t mu, const void* h, int64_t ld, const double* omega, int64_t n_omega,
                         double eta, double* omega_out, double* osc, double* im_eps) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !h || !omega_out || !osc || (n_omega > 0 && (!omega || !im_eps))) return fail(BSE_EINVAL, "null argument");
    if (!(eta > 0)) return fail(BSE_EINVAL, "eta must be positive");
    BSE_TRY(ensure_partner(c, mu));
    auto& pd = c->partner[mu];
    return spectrum_generic(c, pd.part, pd.d, pd.d, !c->t.bright[mu], h, ld, omega, n_omega, eta, omega_out, osc,
                            im_eps);
}

int bse_block_spectrum_lanczos(bse_ctx* c, int32_t mu, int32_t partner, const void* h, int64_t ld, int32_t steps,
                               const double* omega, int64_t n_omega, double eta, double* ritz, double* weights,
                               double* im_eps, int32_t* steps_done) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!h || !steps_done || (!ritz) != (!weights) || (n_omega > 0 && (!omega || !im_eps)))
        return fail(BSE_EINVAL, "null argument");
    if (!(eta > 0)) return fail(BSE_EINVAL, "eta must be positive");
    *steps_done = 0;
    IrrepDev* parts = nullptr;
    int nparts = 1;
    if (partner) {
        BSE_TRY(ensure_partner(c, mu));
        parts = c->partner[mu].part;
        nparts = c->partner[mu].d;
    } else {
        BSE_TRY(ensure_basis(c, mu));
        parts = &c->irr[mu];
    }
    const int64_t dim = parts[0].host.dim;
    if (ld < dim) return fail(BSE_EINVAL, "ld < block dimension");
    if (steps < 1 || steps > std::max<int64_t>(dim, 1))
        return fail(BSE_EINVAL, "steps must be in [1, %lld]", (long long)dim);
    if (ritz) {
        BSE_CUDA(cudaMemsetAsync(ritz, 0, sizeof(double) * steps, c->stream));
        BSE_CUDA(cudaMemsetAsync(weights, 0, sizeof(double) * steps, c->stream));
    }
    if (dim == 0 || !c->t.bright[mu]) {   // no dipole weight: an empty spectrum
        if (n_omega) BSE_CUDA(cudaMemsetAsync(im_eps, 0, sizeof(double) * n_omega, c->stream));
        return BSE_OK;
    }
    BSE_TRY(ensure_dipoles(c));
    BSE_TRY(ensure(c->Bmu, sizeof(double2) * (size_t)dim * nparts));
    for (int p = 0; p < nparts; ++p)
        BSE_TRY(launch_bmu(dev_basis_of(c, parts[p]), (const double2*)c->B.p, (double2*)c->Bmu.p + (size_t)p * dim,
                           c->stream));
    int pmax = 0;
    double scale = 0.0;
    BSE_TRY(start_direction(c, nparts, false, dim, &pmax, &scale));
    if (!(scale > 0.0)) {
        if (n_omega) BSE_CUDA(cudaMemsetAsync(im_eps, 0, sizeof(double) * n_omega, c->stream));
        return BSE_OK;
    }
    const size_t lzb = (lanczos_scratch_bytes(dim, steps) + 255) & ~(size_t)255;
    BSE_TRY(ensure(c->lzScratch, lzb + sizeof(double) * (size_t)steps * steps));
    if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[3], c->stream));
    double *alpha = nullptr, *beta = nullptr;
    int done = 0;
    BSE_TRY(launch_lanczos((const double2*)h, ld, dim, (const double2*)c->Bmu.p + (size_t)pmax * dim, steps,
                           c->lzScratch.p, &alpha, &beta, &done, c->stream, c->wait_polls));
    const double pref = 4.0 * M_PI * c->spin / c->t.nk;
    BSE_TRY(launch_cf_spectrum(alpha, beta + 1, done, scale, omega, n_omega, eta, pref, im_eps, c->stream));
    if (c->timing) BSE_CUDA(cudaEventRecord(c->ev[4], c->stream));
    if (ritz) {   // eigenpairs of T_done (dense symmetric eigensolver; clusters of Ritz values are harmless there)
        double* T = (double*)((char*)c->lzScratch.p + lzb);
        BSE_TRY(launch_tm_dense(alpha, beta + 1, done, T, c->stream));
        if (!c->solver && cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS)
            return fail(BSE_ESOLVER, "cusolverDnCreate failed");
        if (cusolverDnSetStream(c->solver, c->stream) != CUSOLVER_STATUS_SUCCESS)
            return fail(BSE_ESOLVER, "cusolverDnSetStream failed");
        int lwork = 0;
        if (cusolverDnDsyevd_bufferSize(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, done, T, done,
                                        ritz, &lwork) != CUSOLVER_STATUS_SUCCESS)
            return fail(BSE_ESOLVER, "dsyevd buffer size query failed");
        BSE_TRY(ensure(c->eigWork, sizeof(double) * (size_t)std::max(lwork, 1)));
        BSE_TRY(ensure(c->info, sizeof(int)));
        if (cusolverDnDsyevd(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, done, T, done, ritz,
                             (double*)c->eigWork.p, lwork, (int*)c->info.p) != CUSOLVER_STATUS_SUCCESS)
            return fail(BSE_ESOLVER, "dsyevd launch failed");
        BSE_TRY(launch_tm_weights(T, done, scale, weights, c->stream));
        int info = 0;
        BSE_CUDA(cudaMemcpyAsync(&info, c->info.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        BSE_CUDA(cudaStreamSynchronize(c->stream));
        if (info != 0) return fail(BSE_ESOLVER, "dsyevd info = %d", info);
    }
    if (c->timing) {
        BSE_CUDA(cudaEventSynchronize(c->ev[4]));
        BSE_CUDA(cudaEventElapsedTime(&c->stats.ms_eig, c->ev[3], c->ev[4]));
    }
    *steps_done = done;
    return BSE_OK;
}

int bse_loss_spectrum(bse_ctx* c, int64_t n, const double* omega_levels, const double* osc, const double* omega,
                      int64_t n_omega, double eta, double* omega_long, double* osc_long, double* loss) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (n < 0 || (n > 0 && (!omega_levels || !osc || !omega_long || !osc_long)) || (n_omega > 0 && (!omega || !loss)))
        return fail(BSE_EINVAL, "null argument");
    if (!(eta > 0)) return fail(BSE_EINVAL, "eta must be positive");
    if (n > (1 << 20)) return fail(BSE_EUNSUPPORTED, "loss spectrum of more than 2^20 levels");
    const double alpha = 4.0 * M_PI * c->spin / c->t.nk;
    if (n > 0) {
        BSE_TRY(ensure(c->lossScratch, loss_scratch_bytes(n)));
        BSE_TRY(launch_loss_levels(omega_levels, osc, n, alpha, c->lossScratch.p, omega_long, osc_long, c->stream));
    }
    if (n_omega > 0) {
        if (n > 0) BSE_TRY(launch_spectrum(omega_long, osc_long, n, omega, n_omega, eta, alpha, loss, c->stream));
        else BSE_CUDA(cudaMemsetAsync(loss, 0, sizeof(double) * n_omega, c->stream));
    }
    return BSE_OK;
}

int bse_set_solver(bse_ctx* c, int32_t solver) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null argument");
    if (solver != BSE_SOLVER_AUTO && solver != BSE_SOLVER_DENSE && solver != BSE_SOLVER_TRIDIAG &&
        solver != BSE_SOLVER_TRIDIAG_BLOCKED && solver != BSE_SOLVER_TRIDIAG_BLOCKED_DF &&
        solver != BSE_SOLVER_TRIDIAG_TWOSTAGE)
        return fail(BSE_EINVAL, "unknown solver %d", solver);
    c->solver_mode = solver;
    return BSE_OK;
}

int bse_set_wait_limit(bse_ctx* c, int64_t polls) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null argument");
    c->wait_polls = polls < 0 ? -1 : (long)std::min<int64_t>(polls, (int64_t)1 << 40);
    return BSE_OK;
}

int bse_set_seeds(bse_ctx* c, int32_t on) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null argument");
    c->seeds = on != 0;
    return BSE_OK;
}

int bse_set_timing(bse_ctx* c, int32_t on) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null argument");
    if (on && !c->ev[0])
        for (auto& e : c->ev) BSE_CUDA(cudaEventCreate(&e));
    c->timing = on != 0;
    return BSE_OK;
}

int bse_get_stats(bse_ctx* c, bse_stats* out) {
    clear_error();
    if (!c || !out) return fail(BSE_EINVAL, "null argument");
    if (c->timing) BSE_CUDA(cudaStreamSynchronize(c->stream));
    *out = c->stats;
    out->launches = launches_total();
    return BSE_OK;
}

int bse_build_blocks_work(bse_ctx* c, int32_t n, const int32_t* irrep, const int32_t* partner, bse_work* out) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null context");
    AllocStream alloc_on_(c->stream);
    if (!c || !out || n < 0 || (n > 0 && !irrep)) return fail(BSE_EINVAL, "null argument");
    std::vector<const Basis*> bases;
    for (int32_t i = 0; i < n; ++i) {
        if (partner && partner[i]) {
            BSE_TRY(ensure_partner(c, irrep[i]));
            bases.push_back(&c->partner[irrep[i]].part[0].host);
        } else {
            BSE_TRY(ensure_basis(c, irrep[i]));
            bases.push_back(&c->irr[irrep[i]].host);
        }
    }
    const Tables& t = c->t;
    *out = bse_work{};
    int64_t total = 0;
    for (const Basis* bh : bases) total += bh->dim;
    if (total == 0) return BSE_OK;
    std::vector<Batch> batches;
    BSE_TRY(plan_batches(t, bases, arena_budget(), batches, c->seeds));
    auto n_o = [&](const Basis& bh, int64_t j) -> double {
        int o = bh.col_orbit[j];
        return (double)(t.orbit_off[o + 1] - t.orbit_off[o]);
    };
    const double nv = t.nv, nc = t.nc;
    double sum_ng = 0, sum_ng2 = 0, proj = 0, exch_tiles = 0, rot_flops = 0;
    BSE_TRY(ensure(c->counter, sizeof(unsigned long long)));
    BSE_CUDA(cudaMemsetAsync(c->counter.p, 0, sizeof(unsigned long long), c->stream));
    for (const Batch& bt : batches) {
        for (const PairTask& p : bt.tasks) {
            int iq[3];
            for (int a = 0; a < 3; ++a) iq[a] = (t.kidx[3 * p.k + a] - t.kidx[3 * p.kp + a] + t.n[a]) % t.n[a];
            int q = (iq[0] * t.n[1] + iq[1]) * t.n[2] + iq[2];
            double ng = c->ng[q];
            sum_ng += ng;
            sum_ng2 += ng * ng;
        }
        for (size_t i = 0; i < bases.size(); ++i)
            for (int j = bt.tile_off[i]; j < bt.tile_off[i + 1]; ++j) {
                const TileTask& tt = bt.tiles[j];
                double sb = 0, sa = 0;
                for (int64_t x = tt.cb0; x < tt.cb1; ++x) sb += n_o(*bases[i], x);
                for (int64_t x = tt.ca0; x < tt.ca1; ++x) sa += n_o(*bases[i], x);
                double mb = (double)(tt.cb1 - tt.cb0), ma = (double)(tt.ca1 - tt.ca0);
                proj += tt.rows * sb + sa * mb;
                exch_tiles += ma * mb;
            }
        out->k_pairs += (int64_t)(bt.tasks.size() + bt.rots.size());
        out->seeds += (int64_t)bt.tasks.size();
        out->rotated += (int64_t)bt.rots.size();
        out->tiles += (int64_t)bt.tiles.size();
        // rotation: per output element the multiplet terms of both sides, two complex products each
        for (const RotTask& r : bt.rots) {
            double right = 0, left = 0;
            for (int v = 0; v < t.nv; ++v)
                for (int cc = 0; cc < t.nc; ++cc) {
                    right += (double)t.band_mult_size(r.kp, v) * t.band_mult_size(r.kp, t.nv + cc);
                    left += (double)t.band_mult_size(r.k, v) * t.band_mult_size(r.k, t.nv + cc);
                }
            rot_flops += 2.0 * 8.0 * t.B * (right + left);
        }
        BSE_TRY(upload(c->tasks, bt.tasks.data(), bt.tasks.size(), c->stream));
        BSE_TRY(launch_count_overlap(c->S, (const PairTask*)c->tasks.p, (int64_t)bt.tasks.size(),
                                     (unsigned long long*)c->counter.p, c->stream));
        BSE_CUDA(cudaStreamSynchronize(c->stream));
    }
    unsigned long long ov = 0;
    BSE_CUDA(cudaMemcpy(&ov, c->counter.p, sizeof(ov), cudaMemcpyDeviceToHost));
    double pmu = 0;
    for (const Basis* bh : bases)
        for (int64_t i = 0; i < bh->dim; ++i) pmu += n_o(*bh, i);
    out->overlap = (int64_t)ov;
    out->rho = 8.0 * (nc * nc + nv * nv) * (double)ov;
    out->contract = 8.0 * (nv * nv * sum_ng2 + nc * nc * nv * nv * sum_ng);
    out->project = 8.0 * proj;
    out->exchange = 8.0 * (pmu + exch_tiles) * c->ng0;
    out->rotate = rot_flops;
    return BSE_OK;
}

int bse_build_work(bse_ctx* c, int32_t mu, int32_t partner, bse_work* out) {
    return bse_build_blocks_work(c, 1, &mu, &partner, out);
}

int bse_sync(bse_ctx* c) {
    clear_error();
    if (!c) return fail(BSE_EINVAL, "null argument");
    BSE_CUDA(cudaStreamSynchronize(c->stream));
    BSE_CUDA(cudaGetLastError());
    return BSE_OK;
}

}  // extern "C"
