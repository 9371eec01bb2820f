"""Longitudinal excitons and the loss spectrum of the oracle (Sec. III.D,
"Excitonic energies and loss spectrum").

Test infrastructure only (see the package docstring).

With the unmodified Coulomb interaction the divergent G = 0 term of the
exchange returns as a rank-one addition (Eq. epsinv_div): in the product
basis H' = H + alpha B* B^T, here with alpha = 4 pi spin / N_k (B carries
1/sqrt(V_uc), Eq. oscillator; spin and the N_k V_uc normalisation as in the
exchange term 2 K^x, so that the roots below are the zeros of Re eps_M of
the spectrum module).  In the eigenbasis of a block (levels Omega_l,
strengths w_l = |B_l|^2, B_l = a_l^T U^T B) the matrix determinant lemma
turns det(H' - x) = 0 into the secular equation (Eq. secular)

    f(x) = 1 - alpha sum_l w_l / (x - Omega_l) = 0,

one root in each gap between consecutive levels with w_l > 0 and one above
the highest; levels with w_l = 0 stay eigenvalues of H'.  The eigenvectors
follow in closed form (Eq. eigenvec_xi), A'_l ~ conj(B_l) / (Omega_l - x),
so the strength of a longitudinal exciton is
|B'_x|^2 = 1 / (alpha^2 sum_l w_l / (Omega_l - x)^2), and
-Im eps_M^-1(omega) = alpha sum_x |B'_x|^2 [eta/((omega - x)^2 + eta^2)
- eta/((omega + x)^2 + eta^2)] (the loss spectrum, same reading of the
anti-resonant term as Im eps_M).
"""
from __future__ import annotations

import math

import numpy as np


def loss_alpha(inp) -> float:
    return 4.0 * math.pi * inp.spin / inp.nk


def secular_levels(Om, osc, alpha, rel_dark=1e-14):
    """Roots of Eq. secular by bisection on each bracketing interval, the
    strengths of Eq. eigenvec_xi; dark levels (w_l <= rel_dark max w) pass
    through with zero strength.  Returns (levels ascending, strengths)."""
    Om = np.asarray(Om, dtype=np.float64)
    osc = np.asarray(osc, dtype=np.float64)
    bright = osc > rel_dark * max(osc.max(initial=0.0), 1e-300)
    ob, wb = Om[bright], osc[bright]
    order = np.argsort(ob, kind="stable")
    ob, wb = ob[order], wb[order]
    roots, strengths = [], []
    m = len(ob)
    for j in range(m):
        lo = ob[j]
        hi = ob[j + 1] if j + 1 < m else ob[j] + alpha * wb.sum()
        d = ob[j] - ob        # x - Omega_l = d + delta with x = Omega_j + delta
        a, b = 0.0, hi - lo
        for _ in range(200):
            mid = 0.5 * (a + b)
            if mid <= a or mid >= b:
                break
            f = 1.0 - alpha * np.sum(wb / (d + mid))
            if f < 0.0:
                a = mid
            else:
                b = mid
        x = lo + 0.5 * (a + b)
        roots.append(x)
        s2 = np.sum(wb / (x - ob) ** 2)
        strengths.append(1.0 / (alpha ** 2 * s2) if np.isfinite(s2) and s2 > 0 else 0.0)
    levels = np.concatenate([np.array(roots), Om[~bright]])
    w = np.concatenate([np.array(strengths), np.zeros(int((~bright).sum()))])
    o = np.argsort(levels, kind="stable")
    return levels[o], w[o]


def bruteforce_levels(H_mu, b_mu, alpha):
    """Definition: eigenpairs of H_mu + alpha conj(b) b^T in the block basis
    (b = U^T B), strengths |a'^T b|^2 with the reading of Eq. oscillatorA."""
    c = np.conj(b_mu)
    Hp = H_mu + alpha * np.outer(c, np.conj(c))
    Om, a = np.linalg.eigh(Hp)
    return Om, np.abs(a.T @ b_mu) ** 2


def loss_spectrum(inp, Om_l, osc_l, omega, eta):
    alpha = loss_alpha(inp)
    d1 = omega[:, None] - Om_l[None, :]
    d2 = omega[:, None] + Om_l[None, :]
    return alpha * ((eta / (d1 ** 2 + eta ** 2) - eta / (d2 ** 2 + eta ** 2)) @ osc_l)
