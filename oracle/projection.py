"""Symmetry-adapted product basis of the oracle (Sec. III.C of the paper).

Test infrastructure only (see the package docstring).

  * Band rotations Gamma(s)_{kn}^{k'n'} = <phi_k'n' | s phi_kn>, k' = s k,
    restricted to degenerate n' ~ n (Eq. Ts), with the action of Eq. sphi:
    (s phi)(r) = phi(s^{-1} r), i.e. c'(R^{-T} p) = exp(-2 pi i R^{-T}p . t) c(p).
  * Two-particle representation (Eq. Ttilde): s maps |k v c> to
    sum Gamma(s)_{kc}^{k'c'} conj(Gamma(s)_{kv}^{k'v'}) |k' v' c'>.
  * Projector P_mu = d_mu/|S| sum_s chi_mu(s)^* Gamma~(s) (Eq. projection).
  * Basis: P_mu applied to the unit vectors of each orbit; the paper
    orthonormalises by SVD, whose basis is not unique for equal singular
    values, so the canonical basis used here is modified Gram-Schmidt (two
    passes) over the orbit members in ascending order, keeping a vector when
    its residual norm exceeds 1e-6.  The columns form U_mu and
    H_mu = U_mu^dagger H U_mu (Eqs. transformationU, Hblock).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .hamiltonian import Inputs
from .tables import Group, MeshTables, multiplets, orbits

KEEP_TOL = 1e-6


def band_rotation(inp: Inputs, grp: Group, mt: MeshTables, s: int, k: int) -> np.ndarray:
    """Gamma(s) at k as an Nb x Nb matrix G[n', n] = <phi_{sk,n'} | s phi_{kn}>,
    zero between non-degenerate bands."""
    k2 = int(mt.rotk[s, k])
    nkc = int(inp.nkc[k])
    y = inp.gk[k, :nkc] + mt.f(k)[None, :]                    # full vectors at k
    yr = y @ grp.rk[s].T                                      # R^{-T} p
    m2 = np.rint(yr - mt.f(k2)[None, :]).astype(np.int64)
    if np.abs(yr - mt.f(k2) - m2).max() > 1e-9:
        raise ValueError("rotated vector is off the mesh coset")
    j = inp.index_in_sphere(k2, m2)
    if np.any(j < 0):
        raise ValueError("coset sphere is not closed under the operation")
    phase = np.exp(-2j * math.pi * (yr @ grp.tau[s]))
    c_k = inp.coef[k][:, :nkc]                                # [nb, nkc]
    c_k2 = inp.coef[k2][:, j]                                 # value at R^{-T}p
    g = np.conj(c_k2) @ (phase[:, None] * c_k.T)              # [n', n]
    mask = np.zeros_like(g, dtype=bool)
    for lo, hi in ((0, inp.nv), (inp.nv, inp.nb)):
        for m in multiplets(inp.eps[k], lo, hi):
            mask[np.ix_(m, m)] = True
    return np.where(mask, g, 0.0)


def two_particle_rep(inp: Inputs, grp: Group, mt: MeshTables, s: int) -> sp.csr_matrix:
    """Gamma~(s) as a sparse N x N matrix M with M[J, I] = Gamma~(s)_I^J."""
    nv, nc = inp.nv, inp.nc
    rows, cols, vals = [], [], []
    for k in range(inp.nk):
        k2 = int(mt.rotk[s, k])
        g = band_rotation(inp, grp, mt, s, k)
        gv = g[:nv, :nv]
        gc = g[nv:, nv:]
        blk = np.einsum("dc,wv->wdvc", gc, np.conj(gv)).reshape(nv * nc, nv * nc)
        r, c = np.nonzero(blk)
        rows.append(k2 * nv * nc + r)
        cols.append(k * nv * nc + c)
        vals.append(blk[r, c])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(inp.N, inp.N))


class Basis:
    """Characters, projectors and the canonical symmetry-adapted basis."""

    def __init__(self, inp: Inputs, grp: Group, mt: MeshTables):
        self.inp, self.grp, self.mt = inp, grp, mt
        self.chi, self.dims, self.class_of = grp.characters()
        self.reps = [two_particle_rep(inp, grp, mt, s) for s in range(grp.n)]
        self.orbits = orbits(mt, inp.eps, inp.nv, inp.nc)
        self._u = {}

    def projector(self, mu: int) -> sp.csr_matrix:
        out = sp.csr_matrix((self.inp.N, self.inp.N), dtype=np.complex128)
        for s in range(self.grp.n):
            out = out + np.conj(self.chi[mu, s]) * self.reps[s]
        return out * (self.dims[mu] / self.grp.n)

    def bright(self):
        """Irreps contained in the polar-vector representation (chi = Tr A)."""
        vec = self.grp.vector_character()
        mult = (self.chi.astype(np.float64) @ vec) / self.grp.n
        return [mu for mu in range(len(self.dims)) if round(mult[mu]) > 0]

    def basis(self, mu: int):
        """(U_mu as a dense N x dim array, list of (orbit index, columns))."""
        if mu in self._u:
            return self._u[mu]
        P = self.projector(mu).tocsc()
        cols, owner = [], []
        for o, mem in enumerate(self.orbits):
            acc = []
            for j in mem:
                x = P[:, j].toarray()[mem, 0]
                for _ in range(2):
                    for u in acc:
                        x = x - u * np.vdot(u, x)
                nrm = np.linalg.norm(x)
                if nrm > KEEP_TOL:
                    acc.append(x / nrm)
            for u in acc:
                full = np.zeros(self.inp.N, dtype=np.complex128)
                full[mem] = u
                cols.append(full)
                owner.append(o)
        U = np.array(cols).T if cols else np.zeros((self.inp.N, 0), dtype=np.complex128)
        self._u[mu] = (U, np.array(owner, dtype=np.int64))
        return self._u[mu]

    def block_dim_trace(self, mu: int) -> int:
        """dim of the irrep subspace as Tr P_mu (an integer)."""
        return int(round(self.projector(mu).diagonal().sum().real))


def project(U: np.ndarray, H: np.ndarray) -> np.ndarray:
    """H_mu = U^dagger H U."""
    return U.conj().T @ H @ U


# ---------------------------------------------------------------------------
# partner (row) blocks of an irrep contained once in the polar-vector
# representation.  Its matrices are the Cartesian rotations restricted to
# the irrep's Cartesian subspace, so the row projectors
#   P_ij = d/|S| sum_s conj(Gamma_mu(s)_ij) Gamma~(s)
# are available without tables.  Great orthogonality (Sec. III.C.3: the
# blocks H^{mu i}_{mu j} are multiples of the identity) makes
# U_i^dagger H U_i the same matrix for every partner i, with U_i = P_i1 U_1:
# the block H_mu is d_mu copies of it.
# ---------------------------------------------------------------------------

def partner_irrep_matrices(grp, chi_mu, d):
    """Gamma_mu(s) = E^T A(s) E (d x d) with E an orthonormal basis of the
    range of the vector-representation projector d/|S| sum chi A(s), chosen by
    Gram-Schmidt over the Cartesian axes x, y, z in that order."""
    pv = d / grp.n * np.einsum("s,sij->ij", chi_mu.astype(float), grp.cart)
    cols = []
    for a in range(3):
        x = pv[:, a].copy()
        for e in cols:
            x -= e * (e @ x)
        if np.linalg.norm(x) > 1e-8:
            cols.append(x / np.linalg.norm(x))
    if len(cols) != d:
        raise ValueError("irrep is not contained once in the polar-vector representation")
    E = np.array(cols).T
    return np.einsum("ai,sab,bj->sij", E, grp.cart, E)


def commutant_seed(n: int) -> np.ndarray:
    """A fixed symmetric n x n matrix with generic entries from the
    two-dimensional Kronecker sequence with the generalised golden ratios
    (g1, g2) = (0.7548776662466927, 0.5698402909980532):
    X_ab = frac(g1 (a+1) + g2 (b+1)) + frac(g1 (b+1) + g2 (a+1)) - 1.
    Any generic symmetric matrix serves; this one is reproducible."""
    g1, g2 = 0.7548776662466927, 0.5698402909980532
    a = np.arange(1, n + 1, dtype=np.float64)
    x = g1 * a[:, None] + g2 * a[None, :]
    y = x - np.floor(x)
    return y + y.T - 1.0


def _gram_schmidt(cols, keep, tol):
    """Modified Gram-Schmidt (two passes) over the given columns in order,
    keeping a vector when its residual norm exceeds tol, at most `keep`."""
    acc = []
    for x in cols:
        x = np.array(x, dtype=np.float64)
        for _ in range(2):
            for u in acc:
                x = x - u * (u @ x)
        nrm = np.linalg.norm(x)
        if nrm > tol:
            acc.append(x / nrm)
        if len(acc) == keep:
            break
    return np.array(acc).T


def regular_irrep_matrices(grp, chi_mu, d):
    """Real orthogonal matrices of a d-dimensional irrep with real characters
    from the left regular representation R(s) e_b = e_{sb} (|S| x |S|):
      1. P = d/|S| sum_s chi(s) R(s), i.e. P_ab = d/|S| chi(a b^-1), projects
         onto the d copies of the irrep; B = Gram-Schmidt over its columns
         (d^2 of them survive);
      2. C = sum_s R(s) X R(s)^T with X = commutant_seed commutes with every
         R(s), so on range(P) it acts on the multiplicity space only; its
         eigenspaces there are single copies of the irrep, d-fold each;
      3. the lowest one, E = B Y, is made canonical through its projector
         Q = E E^T: Gram-Schmidt over Q e_0, Q e_1, ... gives E';
      4. Gamma(s) = E'^T R(s) E'.
    Raises ValueError when the lowest eigenspace is not separated."""
    G = grp.n
    chi = np.asarray(chi_mu, dtype=np.float64)
    P = d / G * chi[grp.mult[np.arange(G)[:, None], grp.inverse[None, :]]]
    B = _gram_schmidt(P.T, d * d, 1e-6)
    if B.shape[1] != d * d:
        raise ValueError("projector rank is not d^2")
    X = commutant_seed(G)
    C = np.zeros((G, G))
    for s in range(G):
        pinv = grp.mult[grp.inverse[s]]            # a -> s^-1 a
        C += X[np.ix_(pinv, pinv)]
    w, Y = np.linalg.eigh(B.T @ C @ B)
    if not w[d] - w[d - 1] > 1e-8 * max(abs(w).max(), 1.0):
        raise ValueError("degenerate commutant spectrum")
    E = B @ Y[:, :d]
    Q = E @ E.T
    Ec = _gram_schmidt(Q.T, d, 1e-6)
    gam = np.empty((G, d, d))
    for s in range(G):
        gam[s] = Ec[grp.mult[s]].T @ Ec                 # sum_b E'(sb, i) E'(b, j)
    return gam


def irrep_matrices(grp, chi_mu, d):
    """Real orthogonal matrices Gamma_mu(s) of an irrep: by the Cartesian
    route (partner_irrep_matrices) when the irrep is contained once in the
    polar-vector representation, chi itself when d = 1, otherwise from the
    regular representation (regular_irrep_matrices)."""
    try:
        return partner_irrep_matrices(grp, chi_mu, d)
    except ValueError:
        pass
    if d == 1:
        return np.asarray(chi_mu, dtype=np.float64).reshape(-1, 1, 1)
    return regular_irrep_matrices(grp, chi_mu, d)


class PartnerBasis:
    """Canonical basis of partner 1 of an irrep and its transfers."""

    def __init__(self, basis: Basis, mu: int):
        self.b = basis
        grp = basis.grp
        self.d = int(basis.dims[mu])
        self.gam = irrep_matrices(grp, basis.chi[mu], self.d)
        n = basis.inp.N
        self.P = [[sum(self.d / grp.n * np.conj(self.gam[s, i, j]) * basis.reps[s] for s in range(grp.n))
                   for j in range(self.d)] for i in range(self.d)]
        P11 = self.P[0][0].tocsc()
        cols = []
        for mem in basis.orbits:
            acc = []
            for j in mem:
                x = P11[:, j].toarray()[mem, 0]
                for _ in range(2):
                    for u in acc:
                        x = x - u * np.vdot(u, x)
                nrm = np.linalg.norm(x)
                if nrm > KEEP_TOL:
                    acc.append(x / nrm)
            for u in acc:
                full = np.zeros(n, dtype=np.complex128)
                full[mem] = u
                cols.append(full)
        U1 = np.array(cols).T if cols else np.zeros((n, 0), dtype=np.complex128)
        self.U = [U1] + [self.P[i][0] @ U1 for i in range(1, self.d)]


def partner_spectrum(inp, H1, Us, B, omega, eta):
    """Levels of the partner block, oscillator strengths summed over the
    partners, and Im eps_M (equal to the spectrum of the whole block)."""
    from .spectrum import lorentz_sum
    Om, a = np.linalg.eigh(H1)
    osc = sum(np.abs(a.T @ (U.T @ B)) ** 2 for U in Us)
    return Om, osc, lorentz_sum(inp, Om, osc, omega, eta)


def star_basis(inp: Inputs, grp: Group, mt: MeshTables, orbit_list, star: int, weights):
    """The canonical basis columns that live on the orbits of one k star, for
    the operator sum_s weights[s] Gamma~(s) (an irrep projector: d/|S| chi*;
    a row projector: d/|S| conj(Gamma_mu(s)_11)).  Same construction as
    Basis.basis restricted to one star, for sampled checks on large meshes.
    Returns (product indices of the star's rows, [n_rows x n_cols] array)."""
    nv, nc = inp.nv, inp.nc
    ks = [int(k) for k in mt.stars[star]]
    rows = np.concatenate([np.arange(k * nv * nc, (k + 1) * nv * nc) for k in ks])
    pos = {int(I): i for i, I in enumerate(rows)}
    rot = {}
    cols = []
    for mem in orbit_list:
        if int(mem[0]) // (nv * nc) not in ks:
            continue
        loc = {int(I): i for i, I in enumerate(mem)}
        n_o = len(mem)
        P = np.zeros((n_o, n_o), dtype=np.complex128)
        for jj, I in enumerate(mem):
            k, v, c = int(I) // (nv * nc), (int(I) // nc) % nv, int(I) % nc
            vm = [m for m in multiplets(inp.eps[k], 0, nv) if v in m][0]
            cm = [m for m in multiplets(inp.eps[k], nv, nv + nc) if nv + c in m][0]
            for s in range(grp.n):
                if weights[s] == 0:
                    continue
                if (s, k) not in rot:
                    rot[(s, k)] = band_rotation(inp, grp, mt, s, k)
                g = rot[(s, k)]
                k2 = int(mt.rotk[s, k])
                for vp in vm:
                    for cp in cm:
                        J = (k2 * nv + vp) * nc + (cp - nv)
                        P[loc[J], jj] += weights[s] * g[cp, nv + c] * np.conj(g[vp, v])
        acc = []
        for jj in range(n_o):
            x = P[:, jj].copy()
            for _ in range(2):
                for u in acc:
                    x = x - u * np.vdot(u, x)
            nrm = np.linalg.norm(x)
            if nrm > KEEP_TOL:
                acc.append(x / nrm)
        for u in acc:
            full = np.zeros(len(rows), dtype=np.complex128)
            for i, I in enumerate(mem):
                full[pos[int(I)]] = u[i]
            cols.append(full)
    U = np.array(cols).T if cols else np.zeros((len(rows), 0), dtype=np.complex128)
    return rows, U
