"""Pins of the oracle's pair densities and Hamiltonian (Sec. II, III.B).

The pair densities are checked against an independent route (real-space
products of the periodic parts on an FFT grid, no sphere look-ups); the
Hamiltonian against the invariants the paper fixes: Hermiticity (TDA),
commutation with every symmetry operation, K = 0 spectrum."""
import numpy as np
import pytest

from conftest import oracle_case, oracle_h
from oracle import hamiltonian as hm


def rho_fft(d, k, kp, bands, bands_p):
    """rho via FFT of conj(u_kn) u_k'n' (periodic parts on a grid)."""
    n = np.array(d["mesh"])
    idx = np.array(np.unravel_index(np.arange(np.prod(n)), tuple(n))).T
    gk, nkc, coef = d["gk"], d["nk_count"], d["coef"]
    allg = np.concatenate([gk[x, :nkc[x]] for x in range(len(nkc))])
    L = int(2 * (allg.max() - allg.min()) + 3)
    def u(kk, b):
        A = np.zeros((L, L, L), dtype=complex)
        m = gk[kk, :nkc[kk]] % L
        A[m[:, 0], m[:, 1], m[:, 2]] = coef[kk][b, :nkc[kk]]
        return np.fft.ifftn(A) * L ** 3
    iq = (idx[k] - idx[kp]) % n
    q = int(np.ravel_multi_index(tuple(iq), tuple(n)))
    fold = (idx[kp] + iq - idx[k]) // n
    g = d["gq"][q, :d["ng_count"][q]]
    h = (-(g + fold)) % L
    out = np.zeros((len(bands), len(bands_p), len(g)), dtype=complex)
    for i, b in enumerate(bands):
        for j, bp in enumerate(bands_p):
            D = np.fft.fftn(np.conj(u(k, b)) * u(kp, bp)) / L ** 3
            out[i, j] = D[h[:, 0], h[:, 1], h[:, 2]]
    return out


@pytest.mark.parametrize("name", ["si2", "lif4", "mos2_331"])
def test_pair_density_fft_route(name):
    d, inp, grp, mt, b = oracle_case(name)
    rng = np.random.default_rng(3)
    nb = inp.nb
    pairs = [(0, 0), (1, 0), (0, 1), (inp.nk - 1, 1)] + [tuple(rng.integers(0, inp.nk, 2)) for _ in range(4)]
    for k, kp in pairs:
        got, _ = hm.pair_density(inp, mt, int(k), int(kp), range(nb), range(nb))
        ref = rho_fft(d, int(k), int(kp), range(nb), range(nb))
        assert np.abs(got - ref).max() < 1e-12


@pytest.mark.parametrize("name", ["si2", "mos2_331"])
def test_pair_density_orthonormality(name):
    """rho_nn'(k, k; Q = 0) = delta_nn' (orthonormal bands, Sec. III.A)."""
    d, inp, grp, mt, b = oracle_case(name)
    for k in range(inp.nk):
        rho, q = hm.pair_density(inp, mt, k, k, range(inp.nb), range(inp.nb))
        g0 = int(np.nonzero(np.all(inp.gq[0, :inp.ngc[0]] == 0, axis=1))[0][0])
        assert q == 0
        assert np.abs(rho[:, :, g0] - np.eye(inp.nb)).max() < 1e-13


def test_exchange_psd_low_rank():
    d, inp, grp, mt, b = oracle_case("si4")
    kx = hm.exchange_matrix(inp, mt)
    ev = np.linalg.eigvalsh(kx)
    assert ev.min() > -1e-14 * ev.max()
    assert np.sum(ev > 1e-12 * ev.max()) <= int(inp.ngc[0]) - 1


@pytest.mark.parametrize("terms", ["x", "w", "dxw"])
def test_hamiltonian_hermitian_and_symmetric(terms):
    """H is Hermitian (TDA) and commutes with every Gamma~(s)
    (Sec. III.C.3: [H, Gamma~] = 0 makes H block-diagonal)."""
    d, inp, grp, mt, b = oracle_case("si4")
    H = oracle_h("si4", terms)
    scale = np.abs(H).max()
    assert np.abs(H - H.conj().T).max() <= 1e-14 * scale
    for r in b.reps:
        assert np.abs(r @ H - (r.T @ H.T).T).max() <= 1e-12 * scale


def test_noninteracting_spectrum():
    """With K = 0 the eigenvalues are eps_c - eps_v (Eq. BSE-eigval)."""
    d, inp, grp, mt, b = oracle_case("si4")
    H = hm.full_hamiltonian(inp, mt, w_div=0.0, terms="d")
    ev = np.linalg.eigvalsh(H)
    assert np.abs(ev - np.sort(hm.diagonal(inp))).max() < 1e-14


def test_head_only_on_diagonal():
    """W^div enters only the diagonal: H(w_div) - H(0) = -w_div * 1."""
    d, inp, grp, mt, b = oracle_case("si2")
    h1 = hm.full_hamiltonian(inp, mt, w_div=0.3, terms="d")
    h0 = hm.full_hamiltonian(inp, mt, w_div=0.0, terms="d")
    assert np.allclose(h1 - h0, -0.3 * np.eye(inp.N), atol=1e-15)


def _sub_index(inp, ks):
    b = inp.nv * inp.nc
    return np.concatenate([np.arange(k * b, (k + 1) * b) for k in ks])


def _block_cases(mt):
    """Star-pair row/column sets: a diagonal star pair (rows = cols), an
    off-diagonal pair, and one with rows != cols in order and length."""
    st = [list(map(int, s)) for s in mt.stars]
    big = max(range(len(st)), key=lambda a: len(st[a]))
    other = next(a for a in range(len(st)) if a != big and len(st[a]) > 1)
    return [(st[big], st[big]),
            (st[big], st[other]),
            (st[other][::-1] + st[0], st[big][:3])]


@pytest.mark.parametrize("name", ["si4", "mos2_331"])
def test_hamiltonian_block_is_the_full_h_restricted(name):
    """hamiltonian_block (the star-pair sub-block every full-size parity check
    compares against) equals full_hamiltonian's rows and columns of the same
    product indices (Eq. BSE-eigval with the head correction of Eq. Wdiv on
    the diagonal), element by element."""
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    wd = _wdiv_of(name)
    for rows, cols in _block_cases(mt):
        got = hm.hamiltonian_block(inp, mt, rows, cols, wd)
        ref = H[np.ix_(_sub_index(inp, rows), _sub_index(inp, cols))]
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(H).max()


def _wdiv_of(name):
    from conftest import _H
    oracle_h(name)
    return _H[(name, "wdiv")]
