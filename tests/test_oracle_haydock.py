"""Pins of the Lanczos-Haydock oracle against facts that do not depend on
how it is coded: the Gauss-quadrature moment identity of the Lanczos
tridiagonal, exactness at full length, the continued fraction against the
pole sum of its own Ritz pairs, early termination on an invariant subspace,
and convergence to the exact block spectrum of an oracle block."""
import math

import numpy as np
import pytest

from conftest import oracle_case, oracle_h
from oracle import haydock as hk
from oracle import projection as pj
from oracle import spectrum as spc


def _random_hermitian(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return (a + a.conj().T) / 2, rng.normal(size=n) + 1j * rng.normal(size=n)


def test_moments_of_the_tridiagonal():
    """|c|^2 (T_m^p)_00 = c^H H^p c for p < 2m (m-point Gauss quadrature)."""
    H, c = _random_hermitian(40, 1)
    m = 6
    a, b, n2 = hk.lanczos(H, c, m)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    hn = np.linalg.norm(H, 2)
    for p in range(2 * m):
        lhs = n2 * np.linalg.matrix_power(T, p)[0, 0]
        rhs = np.vdot(c, np.linalg.matrix_power(H, p) @ c).real
        assert abs(lhs - rhs) <= 1e-11 * hn ** p * n2, p
    # one moment further the identity no longer holds in general
    p = 2 * m
    lhs = n2 * np.linalg.matrix_power(T, p)[0, 0]
    rhs = np.vdot(c, np.linalg.matrix_power(H, p) @ c).real
    assert abs(lhs - rhs) > 1e-8 * hn ** p * n2


def test_full_length_is_exact():
    """m = n reproduces sum_l |<c, a_l>|^2 / (z - Omega_l) (well-separated spectrum)."""
    n = 10
    rng = np.random.default_rng(2)
    q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    lam = np.arange(n, dtype=float) + 0.3 * rng.random(n)
    H = (q * lam) @ q.conj().T
    c = rng.normal(size=n) + 1j * rng.normal(size=n)
    a, b, n2 = hk.lanczos(H, c, n)
    assert len(a) == n
    w = np.abs(q.conj().T @ c) ** 2
    z = np.linspace(-2, 12, 57) + 0.05j
    exact = (w[None, :] / (z[:, None] - lam[None, :])).sum(axis=1)
    assert np.abs(hk.continued_fraction(a, b, n2, z) - exact).max() <= 1e-9 * np.abs(exact).max()


def test_continued_fraction_is_the_ritz_pole_sum():
    H, c = _random_hermitian(30, 3)
    a, b, n2 = hk.lanczos(H, c, 12)
    th, wt = hk.ritz(a, b, n2)
    assert abs(wt.sum() - n2) <= 1e-12 * n2
    z = np.linspace(-15, 15, 91) + 0.2j
    poles = (wt[None, :] / (z[:, None] - th[None, :])).sum(axis=1)
    assert np.abs(hk.continued_fraction(a, b, n2, z) - poles).max() <= 1e-11 * np.abs(poles).max()


def test_invariant_subspace_stops_early():
    """c in the span of three eigenvectors: three steps, exact spectrum."""
    lam = np.array([0.5, 1.0, 1.7, 2.2, 3.1, 4.0])
    H = np.diag(lam).astype(np.complex128)
    c = np.array([0.3, 0, 1.1j, 0, 0.7, 0], dtype=np.complex128)
    a, b, n2 = hk.lanczos(H, c, 6)
    assert len(a) == 3
    th, wt = hk.ritz(a, b, n2)
    assert np.allclose(th, [0.5, 1.7, 3.1], atol=1e-13)
    assert np.allclose(wt, [0.09, 1.21, 0.49], atol=1e-13)


@pytest.mark.parametrize("name", ["si4", "mos2_331"])
def test_haydock_converges_to_the_block_spectrum(name):
    """The bright block's Haydock spectrum (start vector conj(U^T B)) within
    1e-3 relative L2 of the exact spectrum of the block, and no farther with
    more steps (a small block's Krylov space may be exhausted early)."""
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    B = spc.dipoles(inp, mt)
    mu = b.bright()[0]
    U, _ = b.basis(mu)
    Hm = pj.project(U, H)
    _, _, exact = spc.block_spectrum(inp, Hm, U, B, d["omega"], d["eta"])
    c = np.conj(U.T @ B)
    errs = []
    for m in (8, 40):
        a, bb, n2 = hk.lanczos(Hm, c, m)
        got = hk.haydock_spectrum(inp, a, bb, n2, d["omega"], d["eta"])
        errs.append(np.linalg.norm(got - exact) / np.linalg.norm(exact))
    assert errs[1] <= 1e-3 and errs[1] <= errs[0] * (1 + 1e-6), errs
