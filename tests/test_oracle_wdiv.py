"""Pins of the head correction W^div (Eqs. Wdiv, divergence_int, divergence_sum)."""
import itertools
import math

import numpy as np
from scipy import integrate

from conftest import oracle_case
from oracle import hamiltonian as hm


def test_qmax_relation():
    b = hm.B_DIV
    assert abs(b - math.exp(-b * hm.q_max(b) ** 2)) < 1e-15
    assert abs(hm.q_max(0.005) - 32.5525) < 1e-3


def test_smoothing_function():
    f = hm.smooth
    assert f(-1.0) == 1.0 and f(1.0) == 0.0
    # continuous first derivative at both ends
    assert abs((f(-1 + 1e-6) - f(-1)) / 1e-6) < 1e-5
    assert abs((f(1) - f(1 - 1e-6)) / 1e-6) < 1e-5


def test_integral_isotropic_radial_quadrature():
    eps = 12.0
    b = hm.B_DIV
    ref, _ = integrate.quad(lambda q: 4 * math.pi * math.exp(-b * q * q) / eps, 0.0, hm.q_max(b), limit=200,
                            epsabs=1e-14, epsrel=1e-14)
    assert abs(hm.divergence_integral(eps * np.eye(3)) - ref) < 1e-12 * ref


def test_h00_uniaxial_closed_form():
    """Y_00 coefficient of 1/(q^T L q) for L = diag(a, a, c), c < a:
    int dOmega /(q^T L q) = 4 pi artanh(k)/(a k), k = sqrt((a - c)/a)."""
    a, c = 15.0, 6.0
    kk = math.sqrt((a - c) / a)
    ref = 4 * math.pi * math.atanh(kk) / (a * kk) / math.sqrt(4 * math.pi)
    assert abs(hm.h00(np.diag([a, a, c])) - ref) < 1e-11 * ref
    # isotropic limit
    assert abs(hm.h00(7.0 * np.eye(3)) - math.sqrt(4 * math.pi) / 7.0) < 1e-12


def test_sum_brute_force_small():
    """The vectorised lattice sum equals a plain loop over mesh points for a
    large b (few terms)."""
    d, inp, grp, mt, b = oracle_case("si2")
    bb = 0.5
    qm = hm.q_max(bb)
    delta = (8 * math.pi ** 3 / inp.v_uc / inp.nk) ** (1 / 3)
    L = inp.eps_inf
    n = np.array(inp.mesh)
    tot = 0.0
    r = 12
    for x in itertools.product(range(-r, r + 1), repeat=3):
        if x == (0, 0, 0):
            continue
        Q = inp.recip @ (np.array(x) / n)
        q = math.sqrt(Q @ Q)
        if q > qm + delta:
            continue
        w = 1.0 if q < qm - delta else hm.smooth((q - qm) / delta)
        tot += math.exp(-bb * q * q) / (Q @ L @ Q) * w
    assert abs(hm.divergence_sum(inp, bb) - tot) < 1e-13 * tot


def test_head_correction_limit():
    """For a fine mesh the double-counting sum approaches the integral, so
    W^div shrinks like N_k^{-1/3} (the q = 0 cell has radius ~ Delta)."""
    d, inp, grp, mt, b = oracle_case("si2")
    w2 = hm.head_correction(inp)
    d4, inp4, *_ = oracle_case("si4")
    w4 = hm.head_correction(inp4)
    assert 0 < w4 < w2
    assert abs(w2 / w4 - 2.0) < 0.2


def test_sum_brute_force_uniaxial():
    """The lattice sum with a uniaxial dielectric tensor (Q^T L Q in the
    denominator, Eq. divergence_sum) equals a plain loop over mesh points."""
    d, inp, grp, mt, b = oracle_case("mos2_331_uni")
    L = inp.eps_inf
    assert L[0, 0] != L[2, 2]
    bb = 0.5
    qm = hm.q_max(bb)
    delta = (8 * math.pi ** 3 / inp.v_uc / inp.nk) ** (1 / 3)
    n = np.array(inp.mesh)
    tot = 0.0
    r = 12
    for x in itertools.product(range(-r, r + 1), repeat=3):
        if x == (0, 0, 0):
            continue
        Q = inp.recip @ (np.array(x) / n)
        q = math.sqrt(Q @ Q)
        if q > qm + delta:
            continue
        w = 1.0 if q < qm - delta else hm.smooth((q - qm) / delta)
        tot += math.exp(-bb * q * q) / (Q @ L @ Q) * w
    assert abs(hm.divergence_sum(inp, bb) - tot) < 1e-13 * tot
