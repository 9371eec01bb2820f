"""Symmetry tables of the oracle (Sec. III.C of the paper).

Test infrastructure only (see the package docstring).

Conventions: an operation {R|t} acts on fractional positions as x -> R x + t
and on wave vectors in reciprocal fractional coordinates as y -> R^{-T} y
(Eq. sk with alpha = 0).  The k mesh is Gamma centred, f_k = (i/n1, j/n2,
l/n3), k = (i*n2 + j)*n3 + l.  Product index I = (k*Nv + v)*Nc + c.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def inv_unimodular(r: np.ndarray) -> np.ndarray:
    """Exact inverse of an integer matrix with determinant +-1 (adjugate)."""
    r = [[int(x) for x in row] for row in r]
    det = (r[0][0] * (r[1][1] * r[2][2] - r[1][2] * r[2][1])
           - r[0][1] * (r[1][0] * r[2][2] - r[1][2] * r[2][0])
           + r[0][2] * (r[1][0] * r[2][1] - r[1][1] * r[2][0]))
    if det not in (1, -1):
        raise ValueError("operation matrix is not unimodular")
    adj = np.zeros((3, 3), dtype=np.int64)
    for i in range(3):
        for j in range(3):
            rows = [x for x in range(3) if x != j]
            cols = [x for x in range(3) if x != i]
            minor = r[rows[0]][cols[0]] * r[rows[1]][cols[1]] - r[rows[0]][cols[1]] * r[rows[1]][cols[0]]
            adj[i, j] = minor * (1 if (i + j) % 2 == 0 else -1)
    return adj * det


class Group:
    """The point group S/S_T of the given space-group operations."""

    def __init__(self, rot, tau, lattice):
        self.rot = np.asarray(rot, dtype=np.int64)
        self.tau = np.asarray(tau, dtype=np.float64)
        self.n = len(self.rot)
        self.lattice = np.asarray(lattice, dtype=np.float64)
        # reciprocal action R^{-T}
        self.rk = np.array([inv_unimodular(r).T for r in self.rot])
        # Cartesian rotation A = L R L^{-1}
        linv = np.linalg.inv(self.lattice)
        self.cart = np.array([self.lattice @ r @ linv for r in self.rot])
        key = {tuple(r.ravel()): i for i, r in enumerate(self.rot)}
        if len(key) != self.n:
            raise ValueError("repeated point-group operation")
        self.mult = np.zeros((self.n, self.n), dtype=np.int64)
        for a in range(self.n):
            for b in range(self.n):
                c = key.get(tuple((self.rot[a] @ self.rot[b]).ravel()))
                if c is None:
                    raise ValueError("operations do not close under multiplication")
                self.mult[a, b] = c
                # the translation parts must compose up to a lattice vector
                d = self.rot[a] @ self.tau[b] + self.tau[a] - self.tau[c]
                if np.abs(d - np.round(d)).max() > 1e-9:
                    raise ValueError("translations do not form a space group")
        self.identity = key[tuple(np.eye(3, dtype=np.int64).ravel())]
        self.inverse = np.array([int(np.nonzero(self.mult[a] == self.identity)[0][0])
                                 for a in range(self.n)])

    # -- conjugacy classes ------------------------------------------------
    def classes(self):
        """Conjugacy classes, numbered by their lowest operation index."""
        cls = -np.ones(self.n, dtype=np.int64)
        reps = []
        for g in range(self.n):
            if cls[g] >= 0:
                continue
            members = {int(self.mult[self.mult[h, g], self.inverse[h]]) for h in range(self.n)}
            for m in members:
                cls[m] = len(reps)
            reps.append(g)
        return cls, reps

    def characters(self, seed: int = 12345):
        """Character table by the Burnside-Dixon method.

        The class sums K_i of a finite group span a commutative algebra with
        K_i K_j = sum_k c_ijk K_k.  In an irrep mu, K_i acts as the scalar
        w_mu(i) = |C_i| chi_mu(g_i) / d_mu, so the vector w_mu is a common
        eigenvector of the matrices (A_i)_{jk} = c_ijk.  A random combination
        of the A_i separates the irreps.  d_mu follows from the first
        orthogonality relation, sum_i |C_i| |chi_mu(g_i)|^2 = |S|.

        Returns (chi [n_irreps, n_ops] rounded to integers, dims, class_of).
        Irreps are ordered by (d_mu, then chi over operations ascending).
        """
        cls, reps = self.classes()
        r = len(reps)
        size = np.bincount(cls, minlength=r)
        c = np.zeros((r, r, r))
        for i in range(r):
            for j in range(r):
                # c_ijk: number of (x in C_i, y in C_j) with x y = z, z fixed in C_k
                for x in np.nonzero(cls == i)[0]:
                    for y in np.nonzero(cls == j)[0]:
                        c[i, j, cls[self.mult[x, y]]] += 1
        c /= size[None, None, :]
        rng = np.random.default_rng(seed)
        comb = np.einsum("i,ijk->jk", rng.standard_normal(r), c)
        # rows: w(j) * x = sum_k comb[j,k] w(k)  ->  w is a right eigenvector of comb
        val, vec = np.linalg.eig(comb)
        e = cls[self.identity]
        out = []
        for m in range(r):
            w = vec[:, m] / vec[e, m]
            d2 = self.n / np.sum(np.abs(w) ** 2 / size)
            d = np.sqrt(d2.real)
            chi_cls = d * w / size
            out.append((int(round(d)), chi_cls))
        chi = np.array([[o[1][cls[s]] for s in range(self.n)] for o in out])
        if np.abs(chi.imag).max() > 1e-8:
            raise ValueError("complex characters are not supported")
        chi_r = np.round(chi.real)
        if np.abs(chi.real - chi_r).max() > 1e-6:
            raise ValueError("characters are not integers")
        dims = np.array([o[0] for o in out], dtype=np.int64)
        order = sorted(range(r), key=lambda m: (dims[m],) + tuple(chi_r[m]))
        return chi_r[order].astype(np.int64), dims[order], cls

    def vector_character(self) -> np.ndarray:
        """chi(s) = Tr A(s), the character of the polar-vector representation."""
        return np.round(np.trace(self.cart, axis1=1, axis2=2)).astype(np.int64)


class MeshTables:
    """k mesh, rotated mesh points, stars (representative = lowest index,
    s_k = lowest operation index with s p = k)."""

    def __init__(self, group: Group, mesh):
        self.group = group
        self.n = tuple(int(x) for x in mesh)
        n1, n2, n3 = self.n
        self.nk = n1 * n2 * n3
        self.idx = np.array(list(itertools.product(range(n1), range(n2), range(n3))))
        nops = group.n
        self.rotk = np.zeros((nops, self.nk), dtype=np.int64)
        self.fold = np.zeros((nops, self.nk, 3), dtype=np.int64)
        for s in range(nops):
            for k in range(self.nk):
                f = [Fraction(int(self.idx[k, i]), self.n[i]) for i in range(3)]
                g = [sum(int(group.rk[s][i, j]) * f[j] for j in range(3)) for i in range(3)]
                fl = [x % 1 for x in g]
                ii = [fl[i] * self.n[i] for i in range(3)]
                if any(x.denominator != 1 for x in ii):
                    raise ValueError("mesh is not invariant under the operations")
                k2 = (int(ii[0]) * n2 + int(ii[1])) * n3 + int(ii[2])
                self.rotk[s, k] = k2
                self.fold[s, k] = [int(g[i] - fl[i]) for i in range(3)]
        self.star_of = -np.ones(self.nk, dtype=np.int64)
        self.star_rep = []
        for k in range(self.nk):
            if self.star_of[k] < 0:
                self.star_of[self.rotk[:, k]] = len(self.star_rep)
                self.star_rep.append(k)
        self.star_rep = np.array(self.star_rep, dtype=np.int64)
        self.s_k = np.array([int(np.nonzero(self.rotk[:, self.star_rep[self.star_of[k]]] == k)[0][0])
                             for k in range(self.nk)], dtype=np.int64)
        self.stars = [np.nonzero(self.star_of == a)[0] for a in range(len(self.star_rep))]

    def f(self, k: int) -> np.ndarray:
        return self.idx[k] / np.array(self.n, dtype=np.float64)

    def index(self, i, j, l) -> int:
        n1, n2, n3 = self.n
        return ((i % n1) * n2 + (j % n2)) * n3 + (l % n3)

    def minus(self, k: int, kp: int):
        """Mesh index of q = k - k' and the integer fold f_k' + f_q - f_k."""
        d = self.idx[k] - self.idx[kp]
        q = self.index(*d)
        fold = (self.idx[kp] + self.idx[q] - self.idx[k]) // np.array(self.n)
        return q, fold

    def little_group(self, k: int):
        return np.nonzero(self.rotk[:, k] == k)[0]


def multiplets(eps_k: np.ndarray, lo: int, hi: int, tol: float = 1e-9):
    """Runs of consecutive bands in [lo, hi) with equal energy (|d eps| <= tol Ha)."""
    out, cur = [], [lo]
    for b in range(lo + 1, hi):
        if abs(eps_k[b] - eps_k[cur[-1]]) <= tol:
            cur.append(b)
        else:
            out.append(cur)
            cur = [b]
    out.append(cur)
    return out


def product_index(k, v, c, nv, nc):
    return (k * nv + v) * nc + c


def orbits(mt: MeshTables, eps: np.ndarray, nv: int, nc: int):
    """Orbits of the product basis (Sec. III.C.4): all (k', v', c') with k' in
    the star of k and v', c' in the multiplets of v, c.  Ordered by lowest
    product index; members ascending.  Returns a list of int arrays."""
    nk = mt.nk
    owner = -np.ones(nk * nv * nc, dtype=np.int64)
    out = []
    for k in range(nk):
        vm = multiplets(eps[k], 0, nv)
        cm = multiplets(eps[k], nv, nv + nc)
        for V in vm:
            for C in cm:
                i0 = product_index(k, V[0], C[0] - nv, nv, nc)
                if owner[i0] >= 0:
                    continue
                mem = []
                for k2 in mt.stars[mt.star_of[k]]:
                    if not np.allclose(eps[k2], eps[k], rtol=0, atol=1e-9):
                        raise ValueError("energies differ within a star")
                    for v in V:
                        for c in C:
                            mem.append(product_index(k2, v, c - nv, nv, nc))
                mem = np.array(sorted(mem), dtype=np.int64)
                owner[mem] = len(out)
                out.append(mem)
    order = sorted(range(len(out)), key=lambda o: out[o][0])
    return [out[o] for o in order]
