"""Block eigensolution and optical spectrum of the oracle (Sec. II, III.D).

Test infrastructure only (see the package docstring).

  * B_kvc = (1/sqrt(V_uc)) <phi_kv| -i qhat.grad |phi_kc> / (eps0_c - eps0_v)
    (Eq. oscillator); with plane waves -i grad -> p, so
    B_kvc = sum_p conj(c_kv(p)) (qhat . p) c_kc(p) / (sqrt(V_uc) (eps0_c - eps0_v)),
    where eps0 = eps - scissor on the conduction bands.
  * B_lambda = sum_I A^lambda_I B_I (Eq. oscillatorA, no conjugation); with
    A = U_mu a, B_lambda = a^T (U_mu^T B).
  * Im eps_M(omega) = (4 pi spin / N_k) sum_lambda |B_lambda|^2
    [eta/((omega - Omega)^2 + eta^2) - eta/((omega + Omega)^2 + eta^2)]
    (Eqs. macro_diel and reducible_polar, read with retarded denominators so
    that Im eps_M is odd in omega).
"""
from __future__ import annotations

import math

import numpy as np

from .hamiltonian import Inputs
from .tables import MeshTables


def dipoles(inp: Inputs, mt: MeshTables) -> np.ndarray:
    """B_I for every product index I = (k, v, c)."""
    nv, nc = inp.nv, inp.nc
    out = np.zeros((inp.nk, nv, nc), dtype=np.complex128)
    for k in range(inp.nk):
        nkc = int(inp.nkc[k])
        p = inp.cart(inp.gk[k, :nkc] + mt.f(k)[None, :])
        qp = p @ inp.qhat
        cv = inp.coef[k][:nv, :nkc]
        cc = inp.coef[k][nv:, :nkc]
        mel = np.conj(cv) @ (qp[:, None] * cc.T)              # [v, c]
        de = (inp.eps[k, nv:] - inp.scissor)[None, :] - inp.eps[k, :nv, None]
        out[k] = mel / de / math.sqrt(inp.v_uc)
    return out.reshape(-1)


def block_spectrum(inp: Inputs, H_mu: np.ndarray, U: np.ndarray, B: np.ndarray,
                   omega: np.ndarray, eta: float):
    """(Omega_lambda, |B_lambda|^2, Im eps_M(omega)) of one block."""
    Om, a = np.linalg.eigh(H_mu)
    Bmu = U.T @ B
    bl = a.T @ Bmu
    osc = np.abs(bl) ** 2
    im = lorentz_sum(inp, Om, osc, omega, eta)
    return Om, osc, im


def lorentz_sum(inp: Inputs, Om, osc, omega, eta):
    pref = 4.0 * math.pi * inp.spin / inp.nk
    d1 = omega[:, None] - Om[None, :]
    d2 = omega[:, None] + Om[None, :]
    return pref * ((eta / (d1 ** 2 + eta ** 2) - eta / (d2 ** 2 + eta ** 2)) @ osc)
