"""Pins of the oracle's projection onto irreps (Sec. III.C.4-5)."""
import numpy as np
import pytest

from conftest import oracle_case, oracle_h
from oracle import projection as pj


@pytest.mark.parametrize("name", ["si2", "mos2_331"])
def test_band_rotations_unitary(name):
    d, inp, grp, mt, b = oracle_case(name)
    for s in range(grp.n):
        for k in range(inp.nk):
            g = pj.band_rotation(inp, grp, mt, s, k)
            assert np.abs(g.conj().T @ g - np.eye(inp.nb)).max() < 1e-12


@pytest.mark.parametrize("name", ["si2", "mos2_331"])
def test_two_particle_rep_homomorphism(name):
    """Gamma~(s1) Gamma~(s2) = Gamma~(s1 s2): translations act trivially on
    products (Sec. III.C.1), so Gamma~ is a representation of S/S_T."""
    d, inp, grp, mt, b = oracle_case(name)
    rng = np.random.default_rng(1)
    for _ in range(12):
        s1, s2 = (int(x) for x in rng.integers(0, grp.n, 2))
        lhs = (b.reps[s1] @ b.reps[s2]).toarray()
        rhs = b.reps[grp.mult[s1, s2]].toarray()
        assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("name", ["si2", "mos2_331"])
def test_projectors(name):
    """P_mu^2 = P_mu, sum_mu P_mu = 1, Tr P_mu = dim of the MGS basis (Eq. projection)."""
    d, inp, grp, mt, b = oracle_case(name)
    tot = np.zeros((inp.N, inp.N), dtype=complex)
    n = 0
    for mu in range(len(b.dims)):
        p = b.projector(mu).toarray()
        assert np.abs(p @ p - p).max() < 1e-12
        tot += p
        U, own = b.basis(mu)
        assert U.shape[1] == b.block_dim_trace(mu)
        if U.shape[1]:
            assert np.abs(U.conj().T @ U - np.eye(U.shape[1])).max() < 1e-12
            assert np.abs(p @ U - U).max() < 1e-12
        n += U.shape[1]
    assert np.abs(tot - np.eye(inp.N)).max() < 1e-12
    assert n == inp.N


def test_orbit_size_bound():
    """Orbit dimension <= |S| d_max^2 (Sec. III.C.5) and equals |star| d_v d_c."""
    d, inp, grp, mt, b = oracle_case("si4")
    for mem in b.orbits:
        assert len(mem) <= grp.n * 9
        ks = sorted(set((mem // (inp.nv * inp.nc)).tolist()))
        assert sorted(ks) == sorted(mt.stars[mt.star_of[ks[0]]].tolist())


def test_block_diagonal_and_eigen_union():
    """U^dagger H U is block diagonal over irreps and the union of block
    eigenvalues is the spectrum of H (Eq. Hblock; brute force at 4x4x4)."""
    d, inp, grp, mt, b = oracle_case("si4")
    H = oracle_h("si4")
    Us = [b.basis(mu)[0] for mu in range(len(b.dims))]
    U = np.concatenate(Us, 1)
    Hb = U.conj().T @ H @ U
    o = 0
    for u in Us:
        Hb[o:o + u.shape[1], o:o + u.shape[1]] = 0.0
        o += u.shape[1]
    assert np.abs(Hb).max() < 1e-13 * np.abs(H).max()
    ev = np.sort(np.concatenate([np.linalg.eigvalsh(pj.project(u, H)) for u in Us]))
    assert np.abs(ev - np.linalg.eigvalsh(H)).max() < 1e-13
    # basis-free form: U H_mu U^dagger = P H P
    mu = b.bright()[0]
    p = b.projector(mu).toarray()
    u = Us[mu]
    assert np.abs(u @ pj.project(u, H) @ u.conj().T - p @ H @ p).max() < 1e-13


def test_block_dimension_ratio():
    """The bright block is about d^2/|S| = 9/48 of the full dimension, as in
    the paper's tables (Si: 0.188 at 60^3, Table I)."""
    d, inp, grp, mt, b = oracle_case("si4")
    mu = b.bright()[0]
    r = b.basis(mu)[0].shape[1] / inp.N
    assert 9 / 48 <= r < 0.23
