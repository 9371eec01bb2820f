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
//                  irrep_dim i32[n_irreps], bright i32[n_irreps], orbit_of i32[N]
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

int main(int argc, char** argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s input output\n", argv[0]);
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
    fclose(o);
    return 0;
}
