"""Lanczos-Haydock spectrum of a block (test infrastructure only; see the
package docstring).

Sec. IV names the Lanczos-Haydock method as a way around the diagonalisation
whose absorption spectrum is the sum of the spectra of the contributing
blocks, here the optically active one.  The textbook recurrence from the
start vector c (the dipole projection whose spectral measure Eq. oscillatorA
weighs: |B_lambda|^2 = |<conj(U^T B), a_lambda>|^2):

    v_0 = c / |c|,  beta_0 v_{-1} = 0
    w = H v_j - beta_j v_{j-1},  alpha_j = Re <v_j, w>,  w -= alpha_j v_j,
    beta_{j+1} = |w|,  v_{j+1} = w / beta_{j+1}

without reorthogonalisation.  The m-step tridiagonal T_m gives the
continued fraction

    g_m(z) = |c|^2 / (z - alpha_0 - beta_1^2 / (z - alpha_1 - beta_2^2 / ... (z - alpha_{m-1})))

which approximates g(z) = sum_lambda |B_lambda|^2 / (z - Omega_lambda), and
the spectrum in the convention of Eqs. macro_diel/reducible_polar (read with
retarded denominators):

    Im eps_M(omega) = (4 pi spin / N_k) (-Im g(omega + i eta) + Im g(-omega + i eta)).
"""
from __future__ import annotations

import math

import numpy as np


def lanczos(H: np.ndarray, c: np.ndarray, m: int, tol: float = 1e-14):
    """m steps of the Hermitian Lanczos recurrence from c.  Returns
    (alpha[:k], beta[1:k], |c|^2) with k <= m the steps performed; the
    recurrence stops early when beta_{j+1} <= tol (|alpha_j| + beta_j), an
    invariant subspace."""
    norm2 = float(np.vdot(c, c).real)
    v = c / math.sqrt(norm2)
    v_prev = np.zeros_like(v)
    b = 0.0
    alpha, beta = [], []
    for j in range(m):
        w = H @ v - b * v_prev
        a = float(np.vdot(v, w).real)
        w = w - a * v
        alpha.append(a)
        if j == m - 1:
            break
        b_next = float(np.linalg.norm(w))
        if b_next <= tol * (abs(a) + b):
            break
        beta.append(b_next)
        v_prev, v, b = v, w / b_next, b_next
    return np.array(alpha), np.array(beta), norm2


def continued_fraction(alpha: np.ndarray, beta: np.ndarray, norm2: float, z: np.ndarray) -> np.ndarray:
    """g_m(z) evaluated from the bottom of the fraction up."""
    z = np.asarray(z, dtype=np.complex128)
    t = z - alpha[-1]
    for j in range(len(alpha) - 2, -1, -1):
        t = z - alpha[j] - beta[j] ** 2 / t
    return norm2 / t


def haydock_spectrum(inp, alpha, beta, norm2, omega, eta):
    """Im eps_M(omega) from the continued fraction."""
    pref = 4.0 * math.pi * inp.spin / inp.nk
    omega = np.asarray(omega, dtype=np.float64)
    gp = continued_fraction(alpha, beta, norm2, omega + 1j * eta)
    gm = continued_fraction(alpha, beta, norm2, -omega + 1j * eta)
    return pref * (-gp.imag + gm.imag)


def ritz(alpha, beta, norm2):
    """Eigenvalues theta_k of T_m and the Gauss weights norm2 z_0(k)^2."""
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    th, z = np.linalg.eigh(T)
    return th, norm2 * z[0] ** 2
