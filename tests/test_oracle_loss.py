"""Pins of the loss-spectrum oracle (Eq. secular, Eq. eigenvec_xi): the
secular-equation roots and closed-form strengths against the brute-force
eigenproblem of H + alpha B* B^T, a one-level closed form, interlacing, and
the invariance of the total strength."""
import numpy as np
import pytest

from conftest import oracle_case, oracle_h
from oracle import loss
from oracle.projection import PartnerBasis, project
from oracle.spectrum import dipoles


def test_one_level_closed_form():
    lv, w = loss.secular_levels([0.3], [2.0], 0.5)
    assert abs(lv[0] - (0.3 + 0.5 * 2.0)) <= 1e-15 and abs(w[0] - 2.0) <= 1e-14


def test_two_levels_closed_form():
    """2x2: the roots of (x - a)(x - b) - alpha (w1 (x - b) + w2 (x - a)) = 0."""
    a, b, w1, w2, al = 0.1, 0.25, 0.7, 0.3, 0.2
    lv, w = loss.secular_levels([a, b], [w1, w2], al)
    p = np.poly1d([1.0, -(a + b) - al * (w1 + w2), a * b + al * (w1 * b + w2 * a)])
    assert np.abs(np.sort(p.r) - lv).max() <= 1e-14
    assert abs(w.sum() - (w1 + w2)) <= 1e-14


@pytest.mark.parametrize("name", ["si4", "lif4", "mos2_331"])
def test_secular_matches_bruteforce(name):
    d, inp, grp, mt, b = oracle_case(name)
    H = oracle_h(name)
    B = dipoles(inp, mt)
    al = loss.loss_alpha(inp)
    for mu in b.bright():
        try:
            U = PartnerBasis(b, mu).U[0]
        except ValueError:
            continue
        if U.shape[1] == 0:
            continue
        Hm = project(U, H)
        bm = U.T @ B
        Om, a = np.linalg.eigh(Hm)
        osc = np.abs(a.T @ bm) ** 2
        lv, w = loss.secular_levels(Om, osc, al)
        ref_lv, ref_w = loss.bruteforce_levels(Hm, bm, al)
        scale = np.linalg.norm(B) ** 2   # a block dark for this polarisation has strengths at rounding level
        assert np.abs(lv - ref_lv).max() <= 1e-12 * np.abs(ref_lv).max()
        assert np.abs(w - ref_w).max() <= 1e-10 * scale
        # interlacing and total strength
        assert np.all(lv >= Om - 1e-15)
        assert abs(w.sum() - osc.sum()) <= 1e-10 * scale


def test_dark_levels_pass_through():
    lv, w = loss.secular_levels([0.1, 0.2, 0.3], [1.0, 0.0, 0.5], 0.1)
    assert np.any(np.abs(lv - 0.2) < 1e-15) and w[np.argmin(np.abs(lv - 0.2))] == 0.0
