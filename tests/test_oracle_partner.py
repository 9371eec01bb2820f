"""Pins of the partner (row) blocks against the irrep block (Sec. III.C.3:
H^{mu i}_{mu j} is a multiple of the identity)."""
import numpy as np
import pytest

from conftest import oracle_case, oracle_h
from oracle import projection as pj
from oracle import spectrum as spc


@pytest.mark.parametrize("name", ["si2", "mos2_331"])
def test_irrep_matrices_are_a_representation(name):
    """Every irrep's matrices: a representation with trace chi, and Schur's
    orthogonality relations across all irreps,
    sum_s Gamma^mu_ij(s) Gamma^nu_kl(s) = |S|/d delta_mu,nu delta_ik delta_jl
    (which also makes each one irreducible and orthogonal)."""
    d, inp, grp, mt, b = oracle_case(name)
    gams = [pj.irrep_matrices(grp, b.chi[mu], int(b.dims[mu])) for mu in range(len(b.dims))]
    for mu, g in enumerate(gams):
        assert np.allclose(np.trace(g, axis1=1, axis2=2), b.chi[mu], atol=1e-12)
        for s1 in range(grp.n):
            for s2 in range(grp.n):
                assert np.allclose(g[s1] @ g[s2], g[grp.mult[s1, s2]], atol=1e-12)
    for mu, g in enumerate(gams):
        for nu, h in enumerate(gams):
            got = np.einsum("sij,skl->ijkl", g, h)
            want = 0.0
            if mu == nu:
                dm = g.shape[1]
                want = grp.n / dm * np.einsum("ik,jl->ijkl", np.eye(dm), np.eye(dm))
            assert np.abs(got - want).max() < 1e-11, (mu, nu)


@pytest.mark.parametrize("name", ["si2", "mos2_331"])
def test_regular_route_equivalent_to_cartesian(name):
    """For the polar-vector irreps both routes give equivalent real
    representations: M = sum_s Gamma_reg(s) Gamma_cart(s)^T intertwines them
    and is a multiple of an orthogonal matrix (Schur's lemma)."""
    d, inp, grp, mt, b = oracle_case(name)
    for mu in b.bright():
        dm = int(b.dims[mu])
        if dm == 1:
            continue
        gc = pj.partner_irrep_matrices(grp, b.chi[mu], dm)
        gr = pj.regular_irrep_matrices(grp, b.chi[mu], dm)
        M = np.einsum("sij,skj->ik", gr, gc)
        c = np.trace(M @ M.T) / dm
        assert c > 1e-6
        assert np.abs(M @ M.T - c * np.eye(dm)).max() < 1e-11 * c
        for s in range(grp.n):
            assert np.allclose(gr[s] @ M, M @ gc[s], atol=1e-11)


@pytest.mark.parametrize("name", ["si2", "si4", "mos2_331"])
def test_partner_blocks(name):
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name) if name != "si2" else __import__("oracle.hamiltonian", fromlist=["x"]).full_hamiltonian(
        inp, mt, w_div=0.01)
    for mu in range(len(b.dims)):   # every irrep: Cartesian, one-dimensional and regular-route matrices
        pb = pj.PartnerBasis(b, mu)
        U, _ = b.basis(mu)
        n1 = pb.U[0].shape[1]
        assert n1 * pb.d == U.shape[1]
        p11 = pb.P[0][0].toarray()
        assert np.abs(p11 @ p11 - p11).max() < 1e-12
        assert abs(np.trace(p11).real - n1) < 1e-9
        assert np.abs(sum(pb.P[i][i].toarray() for i in range(pb.d)) - b.projector(mu).toarray()).max() < 1e-12
        if n1 == 0:
            continue
        H1 = pb.U[0].conj().T @ H @ pb.U[0]
        for i in range(pb.d):
            for j in range(pb.d):
                ov = pb.U[i].conj().T @ pb.U[j]
                assert np.abs(ov - (np.eye(n1) if i == j else 0)).max() < 1e-12
                blk = pb.U[i].conj().T @ H @ pb.U[j]
                assert np.abs(blk - (H1 if i == j else 0)).max() < 1e-12 * np.abs(H).max()
        # the irrep block is d copies of the partner block
        ev = np.sort(np.repeat(np.linalg.eigvalsh(H1), pb.d))
        assert np.abs(ev - np.linalg.eigvalsh(pj.project(U, H))).max() < 1e-12


@pytest.mark.parametrize("name", ["si4", "mos2_331"])
def test_partner_spectrum_equals_block_spectrum(name):
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    B = spc.dipoles(inp, mt)
    for mu in b.bright():
        pb = pj.PartnerBasis(b, mu)
        if pb.U[0].shape[1] == 0:
            continue
        H1 = pb.U[0].conj().T @ H @ pb.U[0]
        Om1, osc1, im1 = pj.partner_spectrum(inp, H1, pb.U, B, d["omega"], d["eta"])
        U, _ = b.basis(mu)
        Om, osc, im = spc.block_spectrum(inp, pj.project(U, H), U, B, d["omega"], d["eta"])
        assert abs(osc1.sum() - osc.sum()) <= 1e-12 * np.linalg.norm(B) ** 2
        assert np.linalg.norm(im1 - im) <= 1e-10 * max(np.linalg.norm(im), 1e-300) + 1e-30


def test_star_basis_matches_global_basis():
    """The star-restricted construction used for sampled checks on large
    meshes reproduces the global canonical bases column by column."""
    d, inp, grp, mt, b = oracle_case("si4")
    mu = b.bright()[0]
    U, _ = b.basis(mu)
    pb = pj.PartnerBasis(b, mu)
    for W, w in ((U, b.dims[mu] / grp.n * b.chi[mu].astype(float)),
                 (pb.U[0], pb.d / grp.n * pb.gam[:, 0, 0])):
        col = 0
        for a in range(len(mt.stars)):
            rows, Ua = pj.star_basis(inp, grp, mt, b.orbits, a, w)
            assert np.abs(W[np.ix_(rows, np.arange(col, col + Ua.shape[1]))] - Ua).max() < 1e-12
            col += Ua.shape[1]
        assert col == W.shape[1]
