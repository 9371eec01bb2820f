// Host-side symmetry tables (Sec. III.C of Stöhler, Blügel, Friedrich):
// the point group S/S_T of the space group, the k mesh and its stars, the
// character table (computed, not typed), multiplets, orbits of the product
// basis and the canonical orthonormal basis of each irrep subspace.
#include <unistd.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <functional>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>

#include "internal.h"

namespace bse {

static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
void clear_error() { g_err.clear(); }
const char* last_error() { return g_err.c_str(); }

static void inv3(const double* a, double* out) {
    double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                 a[2] * (a[3] * a[7] - a[4] * a[6]);
    out[0] = (a[4] * a[8] - a[5] * a[7]) / det;
    out[1] = (a[2] * a[7] - a[1] * a[8]) / det;
    out[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    out[3] = (a[5] * a[6] - a[3] * a[8]) / det;
    out[4] = (a[0] * a[8] - a[2] * a[6]) / det;
    out[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    out[6] = (a[3] * a[7] - a[4] * a[6]) / det;
    out[7] = (a[1] * a[6] - a[0] * a[7]) / det;
    out[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

// exact inverse of a unimodular integer matrix; returns false otherwise
static bool inv_unimodular(const int32_t* r, int32_t* out) {
    long det = (long)r[0] * (r[4] * r[8] - r[5] * r[7]) - (long)r[1] * (r[3] * r[8] - r[5] * r[6]) +
               (long)r[2] * (r[3] * r[7] - r[4] * r[6]);
    if (det != 1 && det != -1) return false;
    int32_t adj[9] = {r[4] * r[8] - r[5] * r[7], r[2] * r[7] - r[1] * r[8], r[1] * r[5] - r[2] * r[4],
                      r[5] * r[6] - r[3] * r[8], r[0] * r[8] - r[2] * r[6], r[2] * r[3] - r[0] * r[5],
                      r[3] * r[7] - r[4] * r[6], r[1] * r[6] - r[0] * r[7], r[0] * r[4] - r[1] * r[3]};
    for (int i = 0; i < 9; ++i) out[i] = adj[i] * (int32_t)det;
    return true;
}

int build_group(Tables& t, const bse_system* sys) {
    t.nops = sys->n_ops;
    if (t.nops <= 0 || t.nops > 48 || !sys->rot || !sys->tau)
        return fail(BSE_EINVAL, "n_ops must be in 1..48 with rot and tau given");
    std::memcpy(t.lattice, sys->lattice, sizeof(t.lattice));
    double linv[9];
    inv3(t.lattice, linv);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t.recip[i * 3 + j] = 2.0 * M_PI * linv[j * 3 + i];
    const double* L = t.lattice;
    t.v_uc = std::fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                       L[2] * (L[3] * L[7] - L[4] * L[6]));
    t.rot.assign(sys->rot, sys->rot + 9 * t.nops);
    t.tau.assign(sys->tau, sys->tau + 3 * t.nops);
    t.rk.resize(9 * t.nops);
    t.cart.resize(9 * t.nops);
    for (int s = 0; s < t.nops; ++s) {
        int32_t inv[9];
        if (!inv_unimodular(&t.rot[9 * s], inv))
            return fail(BSE_EINVAL, "operation %d is not unimodular", s);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) t.rk[9 * s + 3 * i + j] = inv[3 * j + i];
        // A = L R L^{-1}
        double lr[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0;
                for (int l = 0; l < 3; ++l) a += L[3 * i + l] * t.rot[9 * s + 3 * l + j];
                lr[3 * i + j] = a;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a = 0;
                for (int l = 0; l < 3; ++l) a += lr[3 * i + l] * linv[3 * l + j];
                t.cart[9 * s + 3 * i + j] = a;
            }
        for (int i = 0; i < 3; ++i) {
            double o = 0;
            for (int j = 0; j < 3; ++j) o += t.cart[9 * s + 3 * i + j] * t.cart[9 * s + 3 * i + j];
            if (std::fabs(o - 1.0) > 1e-9)
                return fail(BSE_ESYMM, "operation %d is not orthogonal in Cartesian space", s);
        }
    }
    std::map<std::vector<int32_t>, int> key;
    for (int s = 0; s < t.nops; ++s) {
        std::vector<int32_t> v(t.rot.begin() + 9 * s, t.rot.begin() + 9 * s + 9);
        if (!key.emplace(v, s).second) return fail(BSE_ESYMM, "operation %d repeats a rotation", s);
    }
    t.mult.assign((size_t)t.nops * t.nops, -1);
    for (int a = 0; a < t.nops; ++a)
        for (int b = 0; b < t.nops; ++b) {
            std::vector<int32_t> p(9);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    int32_t v = 0;
                    for (int l = 0; l < 3; ++l) v += t.rot[9 * a + 3 * i + l] * t.rot[9 * b + 3 * l + j];
                    p[3 * i + j] = v;
                }
            auto it = key.find(p);
            if (it == key.end()) return fail(BSE_ESYMM, "operations do not close (%d*%d)", a, b);
            int c = it->second;
            t.mult[(size_t)a * t.nops + b] = c;
            for (int i = 0; i < 3; ++i) {
                double d = t.tau[3 * a + i] - t.tau[3 * c + i];
                for (int j = 0; j < 3; ++j) d += t.rot[9 * a + 3 * i + j] * t.tau[3 * b + j];
                if (std::fabs(d - std::nearbyint(d)) > 1e-9)
                    return fail(BSE_ESYMM, "translations of %d*%d do not compose", a, b);
            }
        }
    std::vector<int32_t> e = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    auto it = key.find(e);
    if (it == key.end()) return fail(BSE_ESYMM, "identity operation missing");
    t.identity = it->second;
    return BSE_OK;
}

int build_mesh(Tables& t) {
    int n1 = t.n[0], n2 = t.n[1], n3 = t.n[2];
    if (n1 <= 0 || n2 <= 0 || n3 <= 0) return fail(BSE_EINVAL, "mesh dimensions must be positive");
    t.nk = n1 * n2 * n3;
    t.kidx.resize(3 * t.nk);
    for (int i = 0; i < n1; ++i)
        for (int j = 0; j < n2; ++j)
            for (int l = 0; l < n3; ++l) {
                int k = (i * n2 + j) * n3 + l;
                t.kidx[3 * k] = i;
                t.kidx[3 * k + 1] = j;
                t.kidx[3 * k + 2] = l;
            }
    long Nl = std::lcm(std::lcm((long)n1, (long)n2), (long)n3);
    long step[3] = {Nl / n1, Nl / n2, Nl / n3};
    t.rotk.assign((size_t)t.nops * t.nk, -1);
    // k = sum_j x_j b_j / n_j goes to s k with mesh coordinates (M x) mod n,
    // M_ij = rk_ij n_i / n_j: integral exactly when the mesh is invariant (a
    // column j with n_j = 1 never contributes).  Per operation, tables of
    // (M_ij x) mod n_i replace the integer divisions of a direct evaluation.
    const int nmax = std::max(n1, std::max(n2, n3));
    std::vector<int> tab((size_t)9 * nmax);
    for (int s = 0; s < t.nops; ++s) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                long Mij = 0;
                if (t.n[j] > 1) {
                    const long num = (long)t.rk[9 * s + 3 * i + j] * step[j];
                    if (num % step[i] != 0) return fail(BSE_EINVAL, "mesh not invariant under operation %d", s);
                    Mij = num / step[i];
                }
                int* tb = &tab[(size_t)(3 * i + j) * nmax];
                const long mi = ((Mij % t.n[i]) + t.n[i]) % t.n[i];
                long v = 0;
                for (int x = 0; x < t.n[j]; ++x) {
                    tb[x] = (int)v;
                    v += mi;
                    if (v >= t.n[i]) v -= t.n[i];
                }
            }
        int32_t* out = &t.rotk[(size_t)s * t.nk];
        for (int k = 0; k < t.nk; ++k) {
            const int* x = &t.kidx[3 * k];
            int id[3];
            for (int i = 0; i < 3; ++i) {
                int v = tab[(size_t)(3 * i) * nmax + x[0]] + tab[(size_t)(3 * i + 1) * nmax + x[1]] +
                        tab[(size_t)(3 * i + 2) * nmax + x[2]];
                while (v >= t.n[i]) v -= t.n[i];
                id[i] = v;
            }
            out[k] = (id[0] * n2 + id[1]) * n3 + id[2];
        }
    }
    // folds G-bar_i = floor((R^{-T} f_k)_i), exactly: (R^{-T} f_k)_i = sum_j rk_ij x_j step_j / Nl
    t.fold.assign((size_t)t.nops * t.nk * 3, 0);
    for (int s = 0; s < t.nops; ++s)
        for (int k = 0; k < t.nk; ++k)
            for (int i = 0; i < 3; ++i) {
                long num = 0;
                for (int j = 0; j < 3; ++j) num += (long)t.rk[9 * s + 3 * i + j] * t.kidx[3 * k + j] * step[j];
                const long fl = num >= 0 ? num / Nl : -((-num + Nl - 1) / Nl);
                t.fold[((size_t)s * t.nk + k) * 3 + i] = (int32_t)fl;
            }
    t.star_of.assign(t.nk, -1);
    t.star_rep.clear();
    t.stars.clear();
    for (int k = 0; k < t.nk; ++k) {
        if (t.star_of[k] >= 0) continue;
        int a = (int)t.star_rep.size();
        t.star_rep.push_back(k);
        std::vector<int32_t> mem;
        for (int s = 0; s < t.nops; ++s) {
            int k2 = t.rotk[(size_t)s * t.nk + k];
            if (t.star_of[k2] < 0) {
                t.star_of[k2] = a;
                mem.push_back(k2);
            }
        }
        std::sort(mem.begin(), mem.end());
        t.stars.push_back(mem);
    }
    t.s_k.assign(t.nk, -1);
    t.pos_in_star.assign(t.nk, -1);
    for (size_t a = 0; a < t.stars.size(); ++a) {
        int p = t.star_rep[a];
        for (size_t i = 0; i < t.stars[a].size(); ++i) t.pos_in_star[t.stars[a][i]] = (int)i;
        for (int s = t.nops - 1; s >= 0; --s) t.s_k[t.rotk[(size_t)s * t.nk + p]] = s;
    }
    return BSE_OK;
}

// ---------------------------------------------------------------------------
// characters by the Burnside-Dixon method
// ---------------------------------------------------------------------------

// cyclic Jacobi eigensolver of a real symmetric n x n matrix (row-major).
static void jacobi(std::vector<double>& a, int n, std::vector<double>& v, std::vector<double>& w) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    double nrm = 0;
    for (double x : a) nrm += x * x;
    nrm = std::sqrt(nrm);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        if (std::sqrt(off) <= 1e-15 * nrm) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = a[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
                for (int k = 0; k < n; ++k) {
                    double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

int build_characters(Tables& t) {
    const int G = t.nops;
    std::vector<int32_t> inv(G);
    for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b)
            if (t.mult[(size_t)a * G + b] == t.identity) inv[a] = b;
    t.class_of.assign(G, -1);
    std::vector<int> rep;
    for (int g = 0; g < G; ++g) {
        if (t.class_of[g] >= 0) continue;
        int c = (int)rep.size();
        rep.push_back(g);
        for (int h = 0; h < G; ++h) {
            int x = t.mult[(size_t)t.mult[(size_t)h * G + g] * G + inv[h]];
            t.class_of[x] = c;
        }
    }
    const int r = (int)rep.size();
    std::vector<double> size(r, 0.0);
    for (int g = 0; g < G; ++g) size[t.class_of[g]] += 1.0;
    for (int g = 0; g < G; ++g)
        if (t.class_of[inv[g]] != t.class_of[g])
            return fail(BSE_EUNSUPPORTED, "group is not ambivalent (complex characters)");
    // c[i][j][k] = #{x in C_i, y in C_j: x y = z} for a fixed z in C_k
    std::vector<double> c((size_t)r * r * r, 0.0);
    for (int x = 0; x < G; ++x)
        for (int y = 0; y < G; ++y)
            c[((size_t)t.class_of[x] * r + t.class_of[y]) * r + t.class_of[t.mult[(size_t)x * G + y]]] += 1.0;
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j)
            for (int k = 0; k < r; ++k) c[((size_t)i * r + j) * r + k] /= size[k];
    const int e = t.class_of[t.identity];
    uint64_t state = 0x9E3779B97F4A7C15ull;
    for (int attempt = 0; attempt < 8; ++attempt) {
        // random combination A = sum_i x_i A_i, (A_i)_{jk} = c_ijk; A D is symmetric for
        // ambivalent groups, so S = D^{-1/2} A D^{1/2} is symmetric with eigenvectors D^{-1/2} w.
        std::vector<double> x(r);
        for (int i = 0; i < r; ++i) {
            state = state * 6364136223846793005ull + 1442695040888963407ull;
            x[i] = (double)(state >> 11) / 9007199254740992.0 - 0.5;
        }
        std::vector<double> S((size_t)r * r, 0.0);
        for (int j = 0; j < r; ++j)
            for (int k = 0; k < r; ++k) {
                double a = 0;
                for (int i = 0; i < r; ++i) a += x[i] * c[((size_t)i * r + j) * r + k];
                S[(size_t)j * r + k] = a * std::sqrt(size[k] / size[j]);
            }
        for (int j = 0; j < r; ++j)
            for (int k = j + 1; k < r; ++k)
                if (std::fabs(S[(size_t)j * r + k] - S[(size_t)k * r + j]) > 1e-10)
                    return fail(BSE_EUNSUPPORTED, "class algebra is not symmetric");
        std::vector<double> V, W;
        jacobi(S, r, V, W);
        std::vector<double> sw = W;
        std::sort(sw.begin(), sw.end());
        bool sep = true;
        for (int i = 1; i < r; ++i)
            if (sw[i] - sw[i - 1] < 1e-7) sep = false;
        if (!sep) continue;
        struct Irr { int d; std::vector<int32_t> chi; };
        std::vector<Irr> irr;
        bool ok = true;
        for (int m = 0; m < r && ok; ++m) {
            std::vector<double> w(r);
            for (int j = 0; j < r; ++j) w[j] = V[(size_t)j * r + m] * std::sqrt(size[j]);
            double we = w[e];
            for (int j = 0; j < r; ++j) w[j] /= we;
            double s2 = 0;
            for (int j = 0; j < r; ++j) s2 += w[j] * w[j] / size[j];
            double d = std::sqrt(G / s2);
            Irr ir;
            ir.d = (int)std::lround(d);
            if (std::fabs(d - ir.d) > 1e-6) ok = false;
            ir.chi.resize(G);
            for (int g = 0; g < G; ++g) {
                double ch = d * w[t.class_of[g]] / size[t.class_of[g]];
                long rc = std::lround(ch);
                if (std::fabs(ch - rc) > 1e-6) ok = false;
                ir.chi[g] = (int32_t)rc;
            }
            irr.push_back(ir);
        }
        if (!ok) return fail(BSE_EUNSUPPORTED, "characters are not integers");
        std::sort(irr.begin(), irr.end(), [](const Irr& a, const Irr& b) {
            if (a.d != b.d) return a.d < b.d;
            return a.chi < b.chi;
        });
        t.n_irreps = r;
        t.chi.clear();
        t.irrep_dim.clear();
        for (auto& ir : irr) {
            t.irrep_dim.push_back(ir.d);
            t.chi.insert(t.chi.end(), ir.chi.begin(), ir.chi.end());
        }
        // first orthogonality check and multiplicity in the polar-vector rep
        long sd2 = 0;
        for (int m = 0; m < r; ++m) sd2 += (long)t.irrep_dim[m] * t.irrep_dim[m];
        if (sd2 != G) return fail(BSE_ESYMM, "sum of squared irrep dimensions != |S|");
        t.bright.assign(r, 0);
        for (int m = 0; m < r; ++m) {
            double acc = 0;
            for (int g = 0; g < G; ++g) {
                double tr = t.cart[9 * g] + t.cart[9 * g + 4] + t.cart[9 * g + 8];
                acc += t.chi[(size_t)m * G + g] * tr;
            }
            t.bright[m] = (int32_t)std::lround(acc / G);
        }
        return BSE_OK;
    }
    return fail(BSE_EUNSUPPORTED, "could not separate the irreps");
}

// ---------------------------------------------------------------------------
// multiplets and orbits
// ---------------------------------------------------------------------------
static const double kDegTol = 1e-9;

static void runs(const double* e, int lo, int hi, std::vector<std::pair<int, int>>& out) {
    out.clear();
    int start = lo, last = lo;
    for (int b = lo + 1; b < hi; ++b) {
        if (std::fabs(e[b] - e[last]) <= kDegTol) {
            last = b;
        } else {
            out.emplace_back(start, last - start + 1);
            start = last = b;
        }
    }
    out.emplace_back(start, last - start + 1);
}

int build_multiplets_and_orbits(Tables& t, const double* eps) {
    const int nv = t.nv, nc = t.nc, nb = t.nb;
    t.vmult.resize(t.nk);
    t.cmult.resize(t.nk);
    t.band_mult.assign((size_t)t.nk * nb, -1);
    for (int k = 0; k < t.nk; ++k) {
        runs(eps + (size_t)k * nb, 0, nv, t.vmult[k]);
        runs(eps + (size_t)k * nb, nv, nb, t.cmult[k]);
        int id = 0;
        for (auto& m : t.vmult[k]) {
            for (int b = m.first; b < m.first + m.second; ++b) t.band_mult[(size_t)k * nb + b] = id;
            ++id;
        }
        for (auto& m : t.cmult[k]) {
            for (int b = m.first; b < m.first + m.second; ++b) t.band_mult[(size_t)k * nb + b] = id;
            ++id;
        }
    }
    // energies must be equal across a star (bands map within their multiplet)
    for (int k = 0; k < t.nk; ++k) {
        int p = t.star_rep[t.star_of[k]];
        for (int b = 0; b < nb; ++b)
            if (std::fabs(eps[(size_t)k * nb + b] - eps[(size_t)p * nb + b]) > kDegTol)
                return fail(BSE_ESYMM, "band energies differ within the star of k=%d", k);
    }
    const int64_t N = t.N;
    t.orbit_of.assign(N, -1);
    t.orbit_off.assign(1, 0);
    t.orbit_members.clear();
    t.orbit_star.clear();
    t.orbit_vlo.clear(); t.orbit_vn.clear(); t.orbit_clo.clear(); t.orbit_cn.clear();
    // visiting k in ascending order creates orbits in ascending order of their lowest member
    for (int k = 0; k < t.nk; ++k) {
        if (t.star_rep[t.star_of[k]] != k) continue;
        const auto& st = t.stars[t.star_of[k]];
        for (auto& V : t.vmult[k])
            for (auto& C : t.cmult[k]) {
                int o = (int)t.orbit_star.size();
                t.orbit_star.push_back(t.star_of[k]);
                t.orbit_vlo.push_back(V.first);
                t.orbit_vn.push_back(V.second);
                t.orbit_clo.push_back(C.first - nv);
                t.orbit_cn.push_back(C.second);
                for (int k2 : st)
                    for (int v = V.first; v < V.first + V.second; ++v)
                        for (int c = C.first - nv; c < C.first - nv + C.second; ++c) {
                            int64_t I = ((int64_t)k2 * nv + v) * nc + c;
                            t.orbit_members.push_back(I);
                            t.orbit_of[I] = o;
                        }
                t.orbit_off.push_back((int64_t)t.orbit_members.size());
            }
    }
    for (int64_t I = 0; I < N; ++I)
        if (t.orbit_of[I] < 0) return fail(BSE_ESYMM, "product index %lld has no orbit", (long long)I);
    // order orbits by lowest member: already ascending within a star (k ascending),
    // and stars visited by ascending representative.  Verify.
    for (size_t o = 1; o + 1 < t.orbit_off.size(); ++o)
        if (t.orbit_members[t.orbit_off[o]] < t.orbit_members[t.orbit_off[o - 1]])
            return fail(BSE_ESYMM, "orbit order violated");
    // Gamma layout: per k, the multiplet blocks (valence, then conduction), d x d row-major
    t.gam_koff.assign(t.nk + 1, 0);
    for (int k = 0; k < t.nk; ++k) {
        int64_t n = 0;
        for (auto& m : t.vmult[k]) n += (int64_t)m.second * m.second;
        for (auto& m : t.cmult[k]) n += (int64_t)m.second * m.second;
        t.gam_koff[k + 1] = t.gam_koff[k] + n;
    }
    t.gam_per_s = t.gam_koff[t.nk];
    // position of each band's multiplet block inside Gamma(s) at k
    t.gam_boff.assign((size_t)t.nk * nb, 0);
    for (int k = 0; k < t.nk; ++k) {
        int64_t off = 0;
        for (auto* ms : {&t.vmult[k], &t.cmult[k]})
            for (auto& m : *ms) {
                for (int b = m.first; b < m.first + m.second; ++b) t.gam_boff[(size_t)k * nb + b] = off;
                off += (int64_t)m.second * m.second;
            }
    }
    return BSE_OK;
}

// Host threads for the set-up passes, created on first use and kept for the
// life of the process: a pass over a few hundred small orbits is shorter
// than creating and joining a thread per core.  The workers are detached and
// the pool is never destroyed (no teardown at exit); a forked child builds a
// pool of its own.  One parallel region runs at a time.
namespace {
struct HostPool {
    std::mutex run_mu, mu;
    std::condition_variable cv_start, cv_done;
    const std::function<void(int)>* job = nullptr;
    unsigned gen = 0;
    int want = 0, pending = 0, nworkers = 0;
    pid_t owner = 0;
};

HostPool* host_pool(int nworkers) {
    static std::mutex make_mu;
    static HostPool* pool = nullptr;
    std::lock_guard<std::mutex> lk(make_mu);
    if (!pool || pool->owner != getpid()) {   // first use, or a forked child: a new pool (the old one is left)
        pool = new HostPool();
        pool->owner = getpid();
    }
    while (pool->nworkers < nworkers) {
        const int id = ++pool->nworkers;   // worker ids 1..; the caller is 0
        HostPool* P = pool;
        std::thread([P, id] {
            unsigned seen = 0;
            for (;;) {
                const std::function<void(int)>* job;
                {
                    std::unique_lock<std::mutex> l(P->mu);
                    P->cv_start.wait(l, [&] { return P->gen != seen; });
                    seen = P->gen;
                    if (id >= P->want) continue;
                    job = P->job;
                }
                (*job)(id);
                {
                    std::lock_guard<std::mutex> l(P->mu);
                    if (--P->pending == 0) P->cv_done.notify_all();
                }
            }
        }).detach();
    }
    return pool;
}

// body(w) on nt workers (w = 0 is the calling thread); returns when all are done
void host_run(int nt, const std::function<void(int)>& body) {
    if (nt <= 1) {
        body(0);
        return;
    }
    HostPool* P = host_pool(nt - 1);
    std::lock_guard<std::mutex> run(P->run_mu);
    {
        std::lock_guard<std::mutex> l(P->mu);
        P->job = &body;
        P->want = nt;
        P->pending = nt - 1;
        ++P->gen;
    }
    P->cv_start.notify_all();
    body(0);
    std::unique_lock<std::mutex> l(P->mu);
    P->cv_done.wait(l, [&] { return P->pending == 0; });
}
}  // namespace

// run f(i) for i in [0, n) on the host threads (at most the hardware threads,
// BSE_HOST_THREADS overrides), items taken in order of decreasing cost when
// costs are given so that the largest do not finish last
template <class F>
static void parallel_for(int n, F f, const std::vector<double>* cost = nullptr) {
    int nt = (int)std::thread::hardware_concurrency();
    if (const char* e = std::getenv("BSE_HOST_THREADS")) nt = std::atoi(e);
    nt = std::max(1, std::min(nt, std::min(32, n)));
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    if (cost) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return (*cost)[a] > (*cost)[b]; });
    std::atomic<int> next{0};
    host_run(nt, [&](int) {
        for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) f(order[q]);
    });
}

void host_parallel_for(int n, const std::function<void(int)>& f, const std::vector<double>* cost) {
    parallel_for(n, [&](int i) { f(i); }, cost);
}

int check_band_rotations(const Tables& t) {
    // each multiplet block of Gamma(s) at k must be unitary (one operation per host thread)
    std::atomic<int> bad{-1};
    parallel_for(t.nops, [&](int s) {
        for (int k = 0; k < t.nk && bad.load() < 0; ++k) {
            int64_t off = (int64_t)s * t.gam_per_s + t.gam_koff[k];
            auto chk = [&](const std::vector<std::pair<int, int>>& ms) -> bool {
                for (auto& m : ms) {
                    int d = m.second;
                    const cplx* g = &t.gamma[off];
                    for (int i = 0; i < d; ++i)
                        for (int j = 0; j < d; ++j) {
                            cplx a = 0;
                            for (int l = 0; l < d; ++l) a += std::conj(g[l * d + i]) * g[l * d + j];
                            if (std::abs(a - (i == j ? 1.0 : 0.0)) > 1e-9) return false;
                        }
                    off += (int64_t)d * d;
                }
                return true;
            };
            if (!chk(t.vmult[k]) || !chk(t.cmult[k])) {
                int none = -1;
                bad.compare_exchange_strong(none, s * t.nk + k);
            }
        }
    });
    if (bad.load() >= 0)
        return fail(BSE_ESYMM, "band rotation of operation %d at k=%d is not unitary", bad.load() / t.nk,
                    bad.load() % t.nk);
    return BSE_OK;
}

// Dense restriction to orbit o of P = sum_s w[s] Gamma~(s), column-major
// (column jj = P e_I for the orbit's member jj).  Gamma~(s) maps |k v c> to
// sum Gamma(s)_{kc}^{sk c'} conj(Gamma(s)_{kv}^{sk v'}) |sk v' c'> (Eq. Ttilde).
static void orbit_matrix(const Tables& t, int o, const double* w, std::vector<cplx>& M) {
    const int nv = t.nv, nc = t.nc, nb = t.nb;
    const int vn = t.orbit_vn[o], cn = t.orbit_cn[o], vlo = t.orbit_vlo[o], clo = t.orbit_clo[o];
    const int blk = vn * cn;
    const int64_t m0 = t.orbit_off[o], n_o = t.orbit_off[o + 1] - m0;
    M.assign((size_t)n_o * n_o, cplx(0.0));
    for (int64_t jj = 0; jj < n_o; ++jj) {
        const int64_t I = t.orbit_members[m0 + jj];
        const int k = (int)(I / (nv * nc));
        const int v = (int)((I / nc) % nv), c = (int)(I % nc);
        cplx* col = &M[(size_t)jj * n_o];
        const int64_t ov = t.gam_koff[k] + t.gam_boff[(size_t)k * nb + v];
        const int64_t oc = t.gam_koff[k] + t.gam_boff[(size_t)k * nb + nv + c];
        for (int s = 0; s < t.nops; ++s) {
            if (w[s] == 0.0) continue;
            const int k2 = t.rotk[(size_t)s * t.nk + k];
            const int64_t base = (int64_t)t.pos_in_star[k2] * blk;
            const cplx* gvb = &t.gamma[(size_t)s * t.gam_per_s + ov];   // vn x vn, [v'][v]
            const cplx* gcb = &t.gamma[(size_t)s * t.gam_per_s + oc];   // cn x cn, [c'][c]
            for (int vp = 0; vp < vn; ++vp) {
                const cplx gv = gvb[vp * vn + (v - vlo)];
                if (gv == 0.0) continue;
                const cplx wg = w[s] * std::conj(gv);
                for (int cp = 0; cp < cn; ++cp) col[base + vp * cn + cp] += wg * gcb[cp * cn + (c - clo)];
            }
        }
    }
}

// Column jj of that restriction alone (P e_I for the orbit's member jj), into col[0, n_o).
static void orbit_column(const Tables& t, int o, const double* w, int64_t jj, cplx* col) {
    const int nv = t.nv, nc = t.nc, nb = t.nb;
    const int vn = t.orbit_vn[o], cn = t.orbit_cn[o], vlo = t.orbit_vlo[o], clo = t.orbit_clo[o];
    const int blk = vn * cn;
    const int64_t m0 = t.orbit_off[o], n_o = t.orbit_off[o + 1] - m0;
    for (int64_t i = 0; i < n_o; ++i) col[i] = 0.0;
    const int64_t I = t.orbit_members[m0 + jj];
    const int k = (int)(I / (nv * nc));
    const int v = (int)((I / nc) % nv), c = (int)(I % nc);
    const int64_t ov = t.gam_koff[k] + t.gam_boff[(size_t)k * nb + v];
    const int64_t oc = t.gam_koff[k] + t.gam_boff[(size_t)k * nb + nv + c];
    for (int s = 0; s < t.nops; ++s) {
        if (w[s] == 0.0) continue;
        const int k2 = t.rotk[(size_t)s * t.nk + k];
        const int64_t base = (int64_t)t.pos_in_star[k2] * blk;
        const cplx* gvb = &t.gamma[(size_t)s * t.gam_per_s + ov];
        const cplx* gcb = &t.gamma[(size_t)s * t.gam_per_s + oc];
        for (int vp = 0; vp < vn; ++vp) {
            const cplx gv = gvb[vp * vn + (v - vlo)];
            if (gv == 0.0) continue;
            const cplx wg = w[s] * std::conj(gv);
            for (int cp = 0; cp < cn; ++cp) col[base + vp * cn + cp] += wg * gcb[cp * cn + (c - clo)];
        }
    }
}

// Tr P on orbit o (its rank, P being a projector that leaves the orbit invariant):
// only the operations fixing the member's k contribute to a diagonal element.
static double orbit_trace(const Tables& t, int o, const double* w) {
    const int nv = t.nv, nc = t.nc, nb = t.nb;
    const int vn = t.orbit_vn[o], cn = t.orbit_cn[o], vlo = t.orbit_vlo[o], clo = t.orbit_clo[o];
    const int64_t m0 = t.orbit_off[o], n_o = t.orbit_off[o + 1] - m0;
    double tr = 0.0;
    for (int64_t jj = 0; jj < n_o; ++jj) {
        const int64_t I = t.orbit_members[m0 + jj];
        const int k = (int)(I / (nv * nc));
        const int v = (int)((I / nc) % nv), c = (int)(I % nc);
        const int64_t ov = t.gam_koff[k] + t.gam_boff[(size_t)k * nb + v];
        const int64_t oc = t.gam_koff[k] + t.gam_boff[(size_t)k * nb + nv + c];
        for (int s = 0; s < t.nops; ++s) {
            if (w[s] == 0.0 || t.rotk[(size_t)s * t.nk + k] != k) continue;
            const cplx gv = t.gamma[(size_t)s * t.gam_per_s + ov + (v - vlo) * vn + (v - vlo)];
            const cplx gc = t.gamma[(size_t)s * t.gam_per_s + oc + (c - clo) * cn + (c - clo)];
            tr += (w[s] * std::conj(gv) * gc).real();
        }
    }
    return tr;
}

// cost estimate of orbit o's work: its dense n_o x n_o restriction
static std::vector<double> orbit_costs(const Tables& t) {
    const int no = (int)t.orbit_star.size();
    std::vector<double> c(no);
    for (int o = 0; o < no; ++o) {
        const double n_o = (double)(t.orbit_off[o + 1] - t.orbit_off[o]);
        c[o] = n_o * n_o;
    }
    return c;
}

// run f(o) for every orbit on the host threads, the largest orbits first
template <class F>
static void for_each_orbit(const Tables& t, F f) {
    const std::vector<double> c = orbit_costs(t);
    parallel_for((int)c.size(), f, &c);
}

// canonical orthonormal basis of the range of P = sum_s w[s] Gamma~(s): P e_j
// over each orbit, then two passes of modified Gram-Schmidt, keeping residuals
// with norm > 1e-6 (the irrep projector of Eq. projection has w = d/|S| chi*).
int build_basis_weighted(const Tables& t, const std::vector<double>& w, Basis& out) {
    out = Basis();
    out.col_off.push_back(0);
    const int nstars = (int)t.stars.size();
    out.star_col.assign(nstars + 1, 0);
    const int no = (int)t.orbit_star.size();
    std::vector<std::vector<cplx>> acc_o(no);
    std::vector<int> nacc_o(no, 0);
    for_each_orbit(t, [&](int o) {
        const int64_t n_o = t.orbit_off[o + 1] - t.orbit_off[o];
        thread_local std::vector<cplx> x;   // scratch kept by each host thread
        x.resize(n_o);
        // the orbit contributes rank = Tr P vectors; the columns after the one that
        // completes them have zero residual, so they are neither formed nor projected
        const long rank = std::lround(orbit_trace(t, o, w.data()));
        std::vector<cplx>& acc = acc_o[o];
        int nacc = 0;
        for (int64_t jj = 0; jj < n_o && nacc < rank; ++jj) {
            orbit_column(t, o, w.data(), jj, x.data());
            for (int pass = 0; pass < 2; ++pass)
                for (int a = 0; a < nacc; ++a) {
                    const cplx* u = &acc[(size_t)a * n_o];
                    cplx d = 0;
                    for (int64_t i = 0; i < n_o; ++i) d += std::conj(u[i]) * x[i];
                    for (int64_t i = 0; i < n_o; ++i) x[i] -= u[i] * d;
                }
            double nrm = 0;
            for (auto& z : x) nrm += std::norm(z);
            nrm = std::sqrt(nrm);
            if (nrm > 1e-6) {
                for (auto& z : x) z /= nrm;
                acc.insert(acc.end(), x.begin(), x.end());
                ++nacc;
            }
        }
        nacc_o[o] = nacc;
    });
    for (int o = 0; o < no; ++o) {
        const int64_t n_o = t.orbit_off[o + 1] - t.orbit_off[o];
        for (int a = 0; a < nacc_o[o]; ++a) {
            out.col_orbit.push_back(o);
            out.coef.insert(out.coef.end(), acc_o[o].begin() + (size_t)a * n_o, acc_o[o].begin() + (size_t)(a + 1) * n_o);
            out.col_off.push_back((int64_t)out.coef.size());
        }
        out.star_col[t.orbit_star[o] + 1] += nacc_o[o];
    }
    out.dim = (int64_t)out.col_orbit.size();
    for (int a = 0; a < nstars; ++a) out.star_col[a + 1] += out.star_col[a];
    for (int64_t j = 1; j < out.dim; ++j)
        if (t.orbit_star[out.col_orbit[j]] < t.orbit_star[out.col_orbit[j - 1]])
            return fail(BSE_ESYMM, "basis columns not grouped by star");
    return BSE_OK;
}

int build_basis(const Tables& t, int mu, Basis& out) {
    if (mu < 0 || mu >= t.n_irreps) return fail(BSE_EINVAL, "irrep %d out of range", mu);
    std::vector<double> w(t.nops);
    for (int s = 0; s < t.nops; ++s) w[s] = (double)t.irrep_dim[mu] / t.nops * t.chi[(size_t)mu * t.nops + s];
    return build_basis_weighted(t, w, out);
}

// Modified Gram-Schmidt (two passes) over the n-vectors cols[j*n .. j*n+n),
// j = 0..m-1 in order, keeping a vector when its residual norm exceeds tol,
// at most `keep` of them; out: the kept vectors, column j at out[j*n].
static int gram_schmidt_real(const std::vector<double>& cols, int n, int m, int keep, double tol,
                             std::vector<double>& out) {
    out.clear();
    int r = 0;
    std::vector<double> x(n);
    for (int j = 0; j < m && r < keep; ++j) {
        for (int i = 0; i < n; ++i) x[i] = cols[(size_t)j * n + i];
        for (int pass = 0; pass < 2; ++pass)
            for (int u = 0; u < r; ++u) {
                const double* e = &out[(size_t)u * n];
                double dt = 0;
                for (int i = 0; i < n; ++i) dt += e[i] * x[i];
                for (int i = 0; i < n; ++i) x[i] -= e[i] * dt;
            }
        double nr = 0;
        for (int i = 0; i < n; ++i) nr += x[i] * x[i];
        nr = std::sqrt(nr);
        if (nr > tol) {
            for (int i = 0; i < n; ++i) out.push_back(x[i] / nr);
            ++r;
        }
    }
    return r;
}

// Gamma_mu(s) = E^T A(s) E for an irrep contained once in the polar-vector
// representation, E an orthonormal basis of the range of d/|S| sum chi(s) A(s)
// chosen by Gram-Schmidt over the axes x, y, z.
static int cartesian_irrep_matrices(const Tables& t, int mu, int d, std::vector<double>& gam) {
    double pv[9] = {0};
    for (int s = 0; s < t.nops; ++s)
        for (int i = 0; i < 9; ++i) pv[i] += (double)d / t.nops * t.chi[(size_t)mu * t.nops + s] * t.cart[9 * s + i];
    std::vector<std::array<double, 3>> E;
    for (int a = 0; a < 3; ++a) {
        std::array<double, 3> x = {pv[a], pv[3 + a], pv[6 + a]};
        for (auto& e : E) {
            double dt = e[0] * x[0] + e[1] * x[1] + e[2] * x[2];
            for (int i = 0; i < 3; ++i) x[i] -= e[i] * dt;
        }
        double nr = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (nr > 1e-8) E.push_back({x[0] / nr, x[1] / nr, x[2] / nr});
    }
    if ((int)E.size() != d) return fail(BSE_ESYMM, "irrep %d: Cartesian subspace has dim %d, not %d", mu, (int)E.size(), d);
    gam.assign((size_t)t.nops * d * d, 0.0);
    for (int s = 0; s < t.nops; ++s)
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double acc = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc += E[i][a] * t.cart[9 * s + 3 * a + b] * E[j][b];
                gam[((size_t)s * d + i) * d + j] = acc;
            }
    return BSE_OK;
}

// Real orthogonal matrices of a d-dimensional irrep (real characters) from
// the left regular representation R(s) e_b = e_{sb}:
//   P_ab = d/|S| chi(a b^-1) projects onto the d copies of the irrep; B is
//   Gram-Schmidt over its columns (d^2 vectors).  C = sum_s R(s) X R(s)^T,
//   X a fixed generic symmetric matrix (two-dimensional Kronecker sequence),
//   commutes with the group, so B^T C B has d eigenvalues, d-fold each, whose
//   eigenspaces are single copies of the irrep.  The lowest one, E, is made
//   canonical through its projector: Gram-Schmidt over (E E^T) e_0, e_1, ...
//   gives E', and Gamma(s) = E'^T R(s) E'.
static int regular_irrep_matrices(const Tables& t, int mu, int d, std::vector<double>& gam) {
    const int G = t.nops, d2 = d * d;
    std::vector<int> inv(G, -1);
    for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b)
            if (t.mult[(size_t)a * G + b] == t.identity) inv[a] = b;
    const int32_t* chi = &t.chi[(size_t)mu * G];
    std::vector<double> P((size_t)G * G), B;
    for (int b = 0; b < G; ++b)
        for (int a = 0; a < G; ++a) P[(size_t)b * G + a] = (double)d / G * chi[t.mult[(size_t)a * G + inv[b]]];
    if (gram_schmidt_real(P, G, G, d2, 1e-6, B) != d2) return fail(BSE_ESYMM, "irrep %d: projector rank is not d^2", mu);
    const double g1 = 0.7548776662466927, g2 = 0.5698402909980532;
    auto frac = [](double x) { return x - std::floor(x); };
    std::vector<double> X((size_t)G * G), C((size_t)G * G, 0.0);
    for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b)
            X[(size_t)a * G + b] = frac(g1 * (a + 1) + g2 * (b + 1)) + frac(g1 * (b + 1) + g2 * (a + 1)) - 1.0;
    for (int s = 0; s < G; ++s) {
        const int32_t* row = &t.mult[(size_t)inv[s] * G];   // a -> s^-1 a
        for (int a = 0; a < G; ++a)
            for (int b = 0; b < G; ++b) C[(size_t)a * G + b] += X[(size_t)row[a] * G + row[b]];
    }
    std::vector<double> CB((size_t)G * d2, 0.0), M((size_t)d2 * d2, 0.0), V, W;
    for (int j = 0; j < d2; ++j)
        for (int a = 0; a < G; ++a) {
            double acc = 0;
            for (int b = 0; b < G; ++b) acc += C[(size_t)a * G + b] * B[(size_t)j * G + b];
            CB[(size_t)j * G + a] = acc;
        }
    for (int i = 0; i < d2; ++i)
        for (int j = 0; j < d2; ++j) {
            double acc = 0;
            for (int a = 0; a < G; ++a) acc += B[(size_t)i * G + a] * CB[(size_t)j * G + a];
            M[(size_t)i * d2 + j] = acc;
        }
    jacobi(M, d2, V, W);
    std::vector<int> order(d2);
    for (int i = 0; i < d2; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return W[x] < W[y]; });
    double wmax = 1.0;
    for (double w : W) wmax = std::max(wmax, std::fabs(w));
    if (!(W[order[d]] - W[order[d - 1]] > 1e-8 * wmax))
        return fail(BSE_ESYMM, "irrep %d: degenerate commutant spectrum", mu);
    std::vector<double> E((size_t)G * d, 0.0), Q((size_t)G * G, 0.0), Ec;
    for (int c = 0; c < d; ++c)
        for (int j = 0; j < d2; ++j) {
            const double y = V[(size_t)j * d2 + order[c]];   // eigenvector order[c], component j
            for (int a = 0; a < G; ++a) E[(size_t)c * G + a] += B[(size_t)j * G + a] * y;
        }
    for (int b = 0; b < G; ++b)
        for (int a = 0; a < G; ++a) {
            double acc = 0;
            for (int c = 0; c < d; ++c) acc += E[(size_t)c * G + a] * E[(size_t)c * G + b];
            Q[(size_t)b * G + a] = acc;
        }
    if (gram_schmidt_real(Q, G, G, d, 1e-6, Ec) != d) return fail(BSE_ESYMM, "irrep %d: eigenspace rank is not d", mu);
    gam.assign((size_t)G * d * d, 0.0);
    for (int s = 0; s < G; ++s)
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double acc = 0;
                for (int b = 0; b < G; ++b) acc += Ec[(size_t)i * G + t.mult[(size_t)s * G + b]] * Ec[(size_t)j * G + b];
                gam[((size_t)s * d + i) * d + j] = acc;
            }
    return BSE_OK;
}

// Real orthogonal matrices Gamma_mu(s) of irrep mu: the Cartesian route for
// an irrep contained once in the polar-vector representation, chi itself for
// a one-dimensional irrep, the regular-representation route otherwise.  The
// result is checked: a representation with trace chi.
int partner_matrices(const Tables& t, int mu, int& d, std::vector<double>& gam) {
    if (mu < 0 || mu >= t.n_irreps) return fail(BSE_EINVAL, "irrep %d out of range", mu);
    d = t.irrep_dim[mu];
    const int G = t.nops;
    if (t.bright[mu] == 1) {
        BSE_TRY(cartesian_irrep_matrices(t, mu, d, gam));
    } else if (d == 1) {
        gam.resize(G);
        for (int s = 0; s < G; ++s) gam[s] = t.chi[(size_t)mu * G + s];
    } else {
        BSE_TRY(regular_irrep_matrices(t, mu, d, gam));
    }
    for (int s1 = 0; s1 < G; ++s1) {
        double tr = 0;
        for (int i = 0; i < d; ++i) tr += gam[((size_t)s1 * d + i) * d + i];
        if (std::fabs(tr - t.chi[(size_t)mu * G + s1]) > 1e-9) return fail(BSE_ESYMM, "irrep %d: trace is not chi", mu);
        for (int s2 = 0; s2 < G; ++s2) {
            const double* g12 = &gam[(size_t)t.mult[(size_t)s1 * G + s2] * d * d];
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    double acc = 0;
                    for (int k = 0; k < d; ++k)
                        acc += gam[((size_t)s1 * d + i) * d + k] * gam[((size_t)s2 * d + k) * d + j];
                    if (std::fabs(acc - g12[i * d + j]) > 1e-9)
                        return fail(BSE_ESYMM, "irrep %d: matrices are not a representation", mu);
                }
        }
    }
    return BSE_OK;
}

// outs[i] columns = (sum_s ws[i][s] Gamma~(s)) u, column by column (orbit-local),
// for every i in one pass over the orbits
int transfer_bases(const Tables& t, const Basis& u, const std::vector<std::vector<double>>& ws,
                   const std::vector<Basis*>& outs) {
    for (Basis* b : outs) *b = u;
    const int no = (int)t.orbit_star.size();
    // first column of each orbit in u (columns are grouped by orbit)
    std::vector<int64_t> first(no + 1, -1);
    for (int64_t j = u.dim - 1; j >= 0; --j) first[u.col_orbit[j]] = j;
    std::vector<double> cost = orbit_costs(t);
    for (int o = 0; o < no; ++o) {   // building M and applying it to the orbit's columns
        int64_t nc = 0;
        for (int64_t j = first[o]; first[o] >= 0 && j < u.dim && u.col_orbit[j] == o; ++j) ++nc;
        cost[o] *= (double)(1 + nc);
    }
    parallel_for(no, [&](int o) {
        if (first[o] < 0) return;
        const int64_t n_o = t.orbit_off[o + 1] - t.orbit_off[o];
        thread_local std::vector<cplx> M;   // scratch kept by each host thread
        int64_t j1 = first[o];
        while (j1 < u.dim && u.col_orbit[j1] == o) ++j1;
        for (size_t q = 0; q < ws.size(); ++q) {
            orbit_matrix(t, o, ws[q].data(), M);
            // y_j = M x_j for all of the orbit's columns at once: each column of M is
            // read once (M can be megabytes), the vectors y_j stay in cache
            for (int64_t j = first[o]; j < j1; ++j) {
                cplx* y = &outs[q]->coef[u.col_off[j]];
                for (int64_t i = 0; i < n_o; ++i) y[i] = 0.0;
            }
            for (int64_t jj = 0; jj < n_o; ++jj) {
                const cplx* col = &M[(size_t)jj * n_o];
                for (int64_t j = first[o]; j < j1; ++j) {
                    const cplx xj = u.coef[u.col_off[j] + jj];
                    if (xj == 0.0) continue;
                    cplx* y = &outs[q]->coef[u.col_off[j]];
                    for (int64_t i = 0; i < n_o; ++i) y[i] += col[i] * xj;
                }
            }
        }
    }, &cost);
    return BSE_OK;
}

}  // namespace bse
