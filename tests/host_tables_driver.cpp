// Test driver (not part of the library): builds the host tables of one
// system with the library's own host code (csrc/host_tables.cpp) on the CPU
// and writes them out, so that tests can compare them with the oracle
// without a GPU.
//
// input  (binary): lattice f64[9], n_ops i32, rot i32[9 n_ops], tau f64[3 n_ops],
//                  mesh i32[3], nv i32, nc i32, eps f64[nk (nv + nc)]
// output (binary): nk, n_ops, n_stars, n_irreps i32; N, n_orbits i64;
//                  rotk i32[n_ops nk], star_of i32[nk], star_rep i32[n_stars],
//                  s_k i32[nk], class_of i32[n_ops], chi i32[n_irreps n_ops],
//                  irrep_dim i32[n_irreps], bright i32[n_irreps], orbit_of i32[N],
//                  fold i32[n_ops nk 3]
// With a third and fourth argument (band rotations in, bases out), the
// driver also builds the bases from given band rotations Gamma(s): complex
// f64 [n_ops][gam_per_s] in the library's layout (per k the multiplet blocks,
// valence then conduction, [target][source] row-major), and writes
//   gam_per_s i64, n_orbits i64, orbit_off i64[n_orbits + 1],
//   orbit_members i64[orbit_off[n_orbits]], then per irrep the basis of
//   Eq. projection and the partner bases (d = 0 when there are none):
//   basis, d i32, d bases, each basis as dim i64, col_orbit i32[dim],
//   col_off i64[dim + 1], coef c128[col_off[dim]].
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "internal.h"

using namespace bse;

template <class T>
static bool get(FILE* f, T* p, size_t n) {
    return fread(p, sizeof(T), n, f) == n;
}
template <class T>
static void put(FILE* f, const T* p, size_t n) {
    fwrite(p, sizeof(T), n, f);
}

static void put_basis(FILE* o, const Basis& b) {
    put(o, &b.dim, 1);
    put(o, b.col_orbit.data(), b.col_orbit.size());
    put(o, b.col_off.data(), b.col_off.size());
    put(o, b.coef.data(), b.coef.size());
}

// the bases of every irrep and its partner bases, as the library builds them
// (the partner weights are those of the partner-block path)
static int write_bases(Tables& t, const char* gin, const char* bout) {
    FILE* f = fopen(gin, "rb");
    if (!f) return 2;
    t.gamma.resize((size_t)t.nops * t.gam_per_s);
    const bool ok = get(f, t.gamma.data(), t.gamma.size());
    fclose(f);
    if (!ok) {
        fprintf(stderr, "short band rotations\n");
        return 2;
    }
    if (check_band_rotations(t) != BSE_OK) {
        fprintf(stderr, "band rotations not unitary\n");
        return 1;
    }
    FILE* o = fopen(bout, "wb");
    if (!o) return 2;
    const int64_t norb = (int64_t)t.orbit_off.size() - 1;
    put(o, &t.gam_per_s, 1);
    put(o, &norb, 1);
    put(o, t.orbit_off.data(), t.orbit_off.size());
    put(o, t.orbit_members.data(), t.orbit_members.size());
    for (int mu = 0; mu < t.n_irreps; ++mu) {
        Basis b;
        if (build_basis(t, mu, b) != BSE_OK) return 1;
        put_basis(o, b);
        int d = 0;
        std::vector<double> gam;
        if (partner_matrices(t, mu, d, gam) != BSE_OK) {
            const int32_t zero = 0;
            put(o, &zero, 1);
            continue;
        }
        const int G = t.nops;
        auto weights = [&](int i, int j) {
            std::vector<double> w(G);
            for (int s = 0; s < G; ++s) w[s] = (double)d / G * gam[((size_t)s * d + i) * d + j];
            return w;
        };
        std::vector<Basis> part(d);
        if (build_basis_weighted(t, weights(0, 0), part[0]) != BSE_OK) return 1;
        std::vector<std::vector<double>> ws;
        std::vector<Basis*> outs;
        for (int i = 1; i < d; ++i) {
            ws.push_back(weights(i, 0));
            outs.push_back(&part[i]);
        }
        if (d > 1 && transfer_bases(t, part[0], ws, outs) != BSE_OK) return 1;
        const int32_t d32 = d;
        put(o, &d32, 1);
        for (const Basis& pb : part) put_basis(o, pb);
    }
    fclose(o);
    return 0;
}

int main(int argc, char** argv) {
    if (argc != 3 && argc != 5) {
        fprintf(stderr, "usage: %s input output [band_rotations bases]\n", argv[0]);
        return 2;
    }
    FILE* f = fopen(argv[1], "rb");
    if (!f) return 2;
    bse_system s{};
    int32_t nops = 0, mesh[3], nv = 0, nc = 0;
    bool ok = get(f, s.lattice, 9) && get(f, &nops, 1);
    std::vector<int32_t> rot(ok ? 9 * (size_t)nops : 0);
    std::vector<double> tau(ok ? 3 * (size_t)nops : 0);
    ok = ok && get(f, rot.data(), rot.size()) && get(f, tau.data(), tau.size()) && get(f, mesh, 3) && get(f, &nv, 1) &&
         get(f, &nc, 1);
    const size_t nk = ok ? (size_t)mesh[0] * mesh[1] * mesh[2] : 0;
    std::vector<double> eps(nk * (nv + nc));
    ok = ok && get(f, eps.data(), eps.size());
    fclose(f);
    if (!ok) {
        fprintf(stderr, "short input\n");
        return 2;
    }
    s.n_ops = nops;
    s.rot = rot.data();
    s.tau = tau.data();
    Tables t;
    t.nv = nv;
    t.nc = nc;
    t.nb = nv + nc;
    t.B = nv * nc;
    for (int i = 0; i < 3; ++i) t.n[i] = mesh[i];
    if (build_group(t, &s) != BSE_OK || build_mesh(t) != BSE_OK) {
        fprintf(stderr, "group or mesh failed\n");
        return 1;
    }
    t.N = (int64_t)t.nk * t.B;
    if (build_characters(t) != BSE_OK || build_multiplets_and_orbits(t, eps.data()) != BSE_OK) {
        fprintf(stderr, "characters or orbits failed\n");
        return 1;
    }
    FILE* o = fopen(argv[2], "wb");
    if (!o) return 2;
    const int32_t head[4] = {t.nk, t.nops, (int32_t)t.stars.size(), t.n_irreps};
    const int64_t head2[2] = {t.N, (int64_t)t.orbit_off.size() - 1};
    put(o, head, 4);
    put(o, head2, 2);
    put(o, t.rotk.data(), t.rotk.size());
    put(o, t.star_of.data(), t.star_of.size());
    put(o, t.star_rep.data(), t.star_rep.size());
    put(o, t.s_k.data(), t.s_k.size());
    put(o, t.class_of.data(), t.class_of.size());
    put(o, t.chi.data(), t.chi.size());
    put(o, t.irrep_dim.data(), t.irrep_dim.size());
    put(o, t.bright.data(), t.bright.size());
    put(o, t.orbit_of.data(), t.orbit_of.size());
    put(o, t.fold.data(), t.fold.size());
    fclose(o);
    return argc == 5 ? write_bases(t, argv[3], argv[4]) : 0;
}
