"""Pins of the oracle's spectrum (Sec. II, III.D)."""
import numpy as np

from conftest import oracle_case, oracle_h
from oracle import hamiltonian as hm
from oracle import projection as pj
from oracle import spectrum as spc


def test_dipole_only_in_bright_block_and_sum_rule():
    """B_mu = U_mu^T B vanishes outside the optically active irrep and the
    total oscillator strength sum |B_lambda|^2 = |B|^2 (Sec. III.D.1)."""
    d, inp, grp, mt, b = oracle_case("si4")
    B = spc.dipoles(inp, mt)
    br = b.bright()
    for mu in range(len(b.dims)):
        bm = b.basis(mu)[0].T @ B
        if mu in br:
            assert np.linalg.norm(bm) > 0.5 * np.linalg.norm(B)
        else:
            assert np.linalg.norm(bm) < 1e-12 * np.linalg.norm(B)
    mu = br[0]
    U = b.basis(mu)[0]
    Om, osc, im = spc.block_spectrum(inp, pj.project(U, oracle_h("si4")), U, B, d["omega"], d["eta"])
    assert abs(osc.sum() - np.linalg.norm(B) ** 2) < 1e-12 * np.linalg.norm(B) ** 2


def test_noninteracting_lorentzians():
    """K = 0: the spectrum is the single-pole Lorentzian sum over product
    states, independent of the eigenvector basis."""
    d, inp, grp, mt, b = oracle_case("si4")
    B = spc.dipoles(inp, mt)
    mu = b.bright()[0]
    U = b.basis(mu)[0]
    H = hm.full_hamiltonian(inp, mt, w_div=0.0, terms="d")
    Om, osc, im = spc.block_spectrum(inp, pj.project(U, H), U, B, d["omega"], d["eta"])
    ref = spc.lorentz_sum(inp, hm.diagonal(inp), np.abs(B) ** 2, d["omega"], d["eta"])
    assert np.abs(im - ref).max() < 1e-10 * np.abs(ref).max()


def test_im_eps_odd_and_positive():
    d, inp, grp, mt, b = oracle_case("si2")
    om = np.linspace(-1.0, 1.0, 201)
    Om = np.array([0.1, 0.2])
    osc = np.array([1.0, 0.5])
    im = spc.lorentz_sum(inp, Om, osc, om, 0.01)
    assert np.allclose(im, -im[::-1], atol=1e-14)
    assert np.all(im[om > 0] > 0)
