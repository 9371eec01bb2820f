"""Electron-hole Hamiltonian of the oracle (Sec. II and III.B of the paper).

Test infrastructure only (see the package docstring).

Plane-wave form of the paper's interaction matrix elements.  With
phi_kn(r) = V^{-1/2} sum_{p in S_k} c_kn(p) exp(i p.r), V = N_k V_uc the
crystal volume, Eq. w_interaction gives, for the exchange term (w = v-bar,
q = 0) and the direct term (w = W, q = k - k'):

  K^x_{kvc,k'v'c'} = 1/V sum_{G != 0} 4 pi/|G|^2 m^k_cv(G) conj(m^k'_c'v'(G)),
      m^k_cv(G) = sum_p conj(c_kc(p + G)) c_kv(p);
  K^d_{kvc,k'v'c'} = 1/V sum_{Q,Q' in S_q} rho_cc'(Q) W_QQ'(q) conj(rho_vv'(Q')),
      rho_nn'(k,k';Q) = sum_{p' in S_k'} conj(c_kn(p' + Q)) c_k'n'(p'),

and H = diag(eps_c - eps_v) + spin * K^x - K^d (Eq. BSE-eigval, spin factor 2
in front of v-bar for a non-magnetic system without spin-orbit coupling).
At q = 0 the head and wings of W are dropped (they integrate to zero or are
replaced, Sec. III.B); the head is replaced on the diagonal by W^div
(Eq. Wdiv with Eqs. divergence_int and divergence_sum), so H_II -= W^div.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

from .tables import MeshTables


class Inputs:
    """Typed view of an input dictionary (see synth.generate)."""

    def __init__(self, d: dict):
        self.d = d
        self.lattice = np.asarray(d["lattice"], dtype=np.float64)
        self.recip = 2.0 * math.pi * np.linalg.inv(self.lattice).T
        self.v_uc = abs(float(np.linalg.det(self.lattice)))
        self.mesh = tuple(int(x) for x in d["mesh"])
        self.nk = int(np.prod(self.mesh))
        self.nv, self.nc = int(d["nv"]), int(d["nc"])
        self.nb = self.nv + self.nc
        self.N = self.nk * self.nv * self.nc
        self.nkc = np.asarray(d["nk_count"])
        self.gk = np.asarray(d["gk"], dtype=np.int64)
        self.coef = np.asarray(d["coef"])
        self.eps = np.asarray(d["eps"])
        self.ngc = np.asarray(d["ng_count"])
        self.gq = np.asarray(d["gq"], dtype=np.int64)
        self.w = np.asarray(d["w"])
        self.eps_inf = np.asarray(d["eps_inf"], dtype=np.float64)
        self.qhat = np.asarray(d["qhat"], dtype=np.float64)
        self.scissor = float(d["scissor"])
        self.spin = int(d["spin_factor"])
        self.volume = self.nk * self.v_uc
        # dense lookup box: index of integer vector m in S_k, or -1
        allg = np.concatenate([self.gk[k, :self.nkc[k]] for k in range(self.nk)])
        self.box_lo = allg.min(0) - 2
        self.box_hi = allg.max(0) + 2
        shape = tuple(self.box_hi - self.box_lo + 1)
        self.box = -np.ones((self.nk,) + shape, dtype=np.int64)
        for k in range(self.nk):
            m = self.gk[k, :self.nkc[k]] - self.box_lo
            self.box[k, m[:, 0], m[:, 1], m[:, 2]] = np.arange(self.nkc[k])

    def index_in_sphere(self, k: int, m: np.ndarray) -> np.ndarray:
        """Position of integer vectors m (shape [..., 3]) in S_k, -1 if absent."""
        x = m - self.box_lo
        inside = np.all((x >= 0) & (m <= self.box_hi), axis=-1)
        x = np.where(inside[..., None], x, 0)
        out = self.box[k, x[..., 0], x[..., 1], x[..., 2]]
        return np.where(inside, out, -1)

    def cart(self, y: np.ndarray) -> np.ndarray:
        """Cartesian wave vector of reciprocal fractional coordinates."""
        return y @ self.recip.T


def pair_density(inp: Inputs, mt: MeshTables, k: int, kp: int, bands, bands_p):
    """rho[n, n', g] = sum_{p' in S_k'} conj(c_kn(p' + Q_g)) c_k'n'(p'),
    Q_g = f_q + gq[q][g] in S_q, q = k - k' (Eq. w_interaction, plane waves).
    Terms with p' + Q outside S_k vanish (the coefficient is zero there)."""
    q, fold = mt.minus(k, kp)
    ng, nkp = int(inp.ngc[q]), int(inp.nkc[kp])
    target = (inp.gk[kp, None, :nkp, :] + inp.gq[q, :ng, None, :] + fold[None, None, :])
    idx = inp.index_in_sphere(k, target)                      # [ng, nkp]
    ck = inp.coef[k][np.asarray(bands)]                       # [n, NK]
    ckp = inp.coef[kp][np.asarray(bands_p)][:, :nkp]          # [n', nkp]
    gath = np.where(idx[None] >= 0, np.conj(ck[:, np.where(idx >= 0, idx, 0)]), 0.0)
    return np.einsum("ngj,mj->nmg", gath, ckp), q


def exchange_vectors(inp: Inputs, mt: MeshTables):
    """P[I, g] = m^k_cv(G_g) for G_g in S_0 (q = 0 sphere), and v-bar(G_g)
    (= 4 pi/|G|^2, 0 at G = 0)."""
    nv, nc = inp.nv, inp.nc
    ng0 = int(inp.ngc[0])
    P = np.zeros((inp.N, ng0), dtype=np.complex128)
    for k in range(inp.nk):
        rho, q = pair_density(inp, mt, k, k, range(nv, nv + nc), range(nv))
        assert q == 0
        # rho[c, v, g] -> rows (k, v, c)
        P[k * nv * nc:(k + 1) * nv * nc] = np.transpose(rho, (1, 0, 2)).reshape(nv * nc, ng0)
    G = inp.cart(inp.gq[0, :ng0].astype(np.float64))
    g2 = np.einsum("gi,gi->g", G, G)
    vbar = np.where(g2 > 0, 4.0 * math.pi / np.where(g2 > 0, g2, 1.0), 0.0)
    return P, vbar


def exchange_matrix(inp: Inputs, mt: MeshTables) -> np.ndarray:
    """Full K^x (without the spin factor)."""
    P, vbar = exchange_vectors(inp, mt)
    return (P * vbar[None, :]) @ P.conj().T / inp.volume


def w_of_q(inp: Inputs, q: int) -> np.ndarray:
    """W_{QQ'}(q) on S_q; at q = 0 the head and wings are set to zero."""
    ng = int(inp.ngc[q])
    w = np.array(inp.w[q, :ng, :ng])
    if q == 0:
        z = np.nonzero(np.all(inp.gq[0, :ng] == 0, axis=1))[0]
        w[z, :] = 0.0
        w[:, z] = 0.0
    return w


def direct_block(inp: Inputs, mt: MeshTables, k: int, kp: int) -> np.ndarray:
    """K^d[(v,c), (v',c')] for one ordered k pair, rows v*Nc + c."""
    nv, nc = inp.nv, inp.nc
    rc, q = pair_density(inp, mt, k, kp, range(nv, nv + nc), range(nv, nv + nc))
    rv, _ = pair_density(inp, mt, k, kp, range(nv), range(nv))
    w = w_of_q(inp, q)
    blk = np.einsum("cdQ,QR,vwR->vcwd", rc, w, np.conj(rv)) / inp.volume
    return blk.reshape(nv * nc, nv * nc)


def direct_matrix(inp: Inputs, mt: MeshTables, rows=None, cols=None) -> np.ndarray:
    """K^d over all ordered pairs (k in rows, k' in cols), default all k."""
    rows = range(inp.nk) if rows is None else rows
    cols = range(inp.nk) if cols is None else cols
    b = inp.nv * inp.nc
    out = np.zeros((len(rows) * b, len(cols) * b), dtype=np.complex128)
    for i, k in enumerate(rows):
        for j, kp in enumerate(cols):
            out[i * b:(i + 1) * b, j * b:(j + 1) * b] = direct_block(inp, mt, k, kp)
    return out


def diagonal(inp: Inputs) -> np.ndarray:
    """eps_ck - eps_vk for every product index I = (k, v, c)."""
    nv = inp.nv
    ev = inp.eps[:, :nv]
    ec = inp.eps[:, nv:]
    return (ec[:, None, :] - ev[:, :, None]).reshape(-1)


# ---------------------------------------------------------------------------
# head correction W^div
# ---------------------------------------------------------------------------

B_DIV = 0.005


def q_max(b: float = B_DIV) -> float:
    """q_max from b = exp(-b q_max^2)."""
    return math.sqrt(-math.log(b) / b)


def h00(L: np.ndarray) -> float:
    """Y_00 coefficient of 1/(q^T L q) (Eq. hinv0): (1/sqrt(4 pi)) times its
    integral over the unit sphere, here by adaptive quadrature."""
    def f(ph, th):
        n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        return math.sin(th) / float(n @ L @ n)
    val, _ = integrate.dblquad(f, 0.0, math.pi, 0.0, 2.0 * math.pi, epsabs=1e-14, epsrel=1e-13)
    return val / math.sqrt(4.0 * math.pi)


def divergence_integral(L: np.ndarray, b: float = B_DIV) -> float:
    """int_{q<q_max} d^3q exp(-b q^2)/(q^2 q^T L q) = pi H00/sqrt(b) erf(sqrt(b) q_max)
    (Eq. divergence_int)."""
    iso = np.allclose(L, L[0, 0] * np.eye(3), rtol=0, atol=0)
    hh = math.sqrt(4.0 * math.pi) / L[0, 0] if iso else h00(L)
    return math.pi * hh / math.sqrt(b) * math.erf(math.sqrt(b) * q_max(b))


def smooth(x):
    """f(x) = (x^3 - 3x + 2)/4 (Eq. divergence_sum)."""
    return (x ** 3 - 3.0 * x + 2.0) / 4.0


def divergence_sum(inp: Inputs, b: float = B_DIV) -> float:
    """Smoothed double-counting sum of Eq. divergence_sum over all nonzero
    points Q = q + G of the k mesh continued through reciprocal space."""
    qm = q_max(b)
    v_bz = 8.0 * math.pi ** 3 / inp.v_uc
    delta = (v_bz / inp.nk) ** (1.0 / 3.0)
    L = inp.eps_inf
    n = np.array(inp.mesh, dtype=np.float64)
    step = inp.recip / n[None, :]                 # Q = step @ X, X integer
    lim = qm + delta
    ext = [int(math.ceil(n[i] * lim * np.linalg.norm(inp.lattice[:, i]) / (2 * math.pi))) + 1
           for i in range(3)]
    x2 = np.arange(-ext[1], ext[1] + 1, dtype=np.float64)
    x3 = np.arange(-ext[2], ext[2] + 1, dtype=np.float64)
    X2, X3 = np.meshgrid(x2, x3, indexing="ij")
    base = X2[..., None] * step[:, 1] + X3[..., None] * step[:, 2]
    parts = []
    for x1 in range(-ext[0], ext[0] + 1):
        Q = base + x1 * step[:, 0]
        q2 = np.einsum("...i,...i->...", Q, Q)
        ql = np.einsum("...i,ij,...j->...", Q, L, Q)
        q = np.sqrt(q2)
        keep = (q2 > 0) & (q <= lim)
        wgt = np.where(q < qm - delta, 1.0, smooth((q - qm) / delta))
        term = np.where(keep, np.exp(-b * q2) * wgt / np.where(keep, ql, 1.0), 0.0)
        parts.append(float(np.sum(term)))
    return math.fsum(parts)


def head_correction(inp: Inputs, b: float = B_DIV) -> float:
    """W^div = (1/(2 pi^2)) * integral - 4 pi/(N_k V_uc) * sum (Eq. Wdiv)."""
    return (divergence_integral(inp.eps_inf, b) / (2.0 * math.pi ** 2)
            - 4.0 * math.pi / (inp.nk * inp.v_uc) * divergence_sum(inp, b))


def full_hamiltonian(inp: Inputs, mt: MeshTables, w_div: float | None = None,
                     terms: str = "dxw") -> np.ndarray:
    """H = diag(eps_c - eps_v) + spin K^x - K^d - W^div 1 over the full product
    basis.  terms selects 'd' (diagonal incl. W^div), 'x' (exchange), 'w'
    (direct)."""
    H = np.zeros((inp.N, inp.N), dtype=np.complex128)
    if "d" in terms:
        wd = head_correction(inp) if w_div is None else w_div
        H[np.diag_indices(inp.N)] += diagonal(inp) - wd
    if "x" in terms:
        H += inp.spin * exchange_matrix(inp, mt)
    if "w" in terms:
        H -= direct_matrix(inp, mt)
    return H


def hamiltonian_block(inp: Inputs, mt: MeshTables, rows, cols, w_div: float) -> np.ndarray:
    """Rows/columns of the full H restricted to product indices of the k
    points in ``rows`` x ``cols`` (ordered as given, each k contributing its
    Nv*Nc products in (v, c) order): the same entries as full_hamiltonian."""
    nv, nc = inp.nv, inp.nc
    b = nv * nc
    H = -direct_matrix(inp, mt, rows, cols)
    P, vbar = exchange_vectors_for(inp, mt, rows)
    Pc, _ = exchange_vectors_for(inp, mt, cols)
    H += inp.spin * (P * vbar[None, :]) @ Pc.conj().T / inp.volume
    dg = diagonal(inp)
    for i, k in enumerate(rows):
        for j, kp in enumerate(cols):
            if k == kp:
                idx = np.arange(b)
                H[i * b + idx, j * b + idx] += dg[k * b:(k + 1) * b] - w_div
    return H


def exchange_vectors_for(inp: Inputs, mt: MeshTables, ks):
    """Rows of the exchange vectors P for the k points ks (see exchange_vectors)."""
    nv, nc = inp.nv, inp.nc
    ng0 = int(inp.ngc[0])
    P = np.zeros((len(ks) * nv * nc, ng0), dtype=np.complex128)
    for i, k in enumerate(ks):
        rho, q = pair_density(inp, mt, k, k, range(nv, nv + nc), range(nv))
        P[i * nv * nc:(i + 1) * nv * nc] = np.transpose(rho, (1, 0, 2)).reshape(nv * nc, ng0)
    G = inp.cart(inp.gq[0, :ng0].astype(np.float64))
    g2 = np.einsum("gi,gi->g", G, G)
    vbar = np.where(g2 > 0, 4.0 * math.pi / np.where(g2 > 0, g2, 1.0), 0.0)
    return P, vbar
