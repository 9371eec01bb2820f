"""Exact crystal geometry for the synthetic inputs.

Everything that decides an integer (which lattice vectors lie inside a cutoff
sphere, which operations belong to the space group, where a rotated k point
lands) is computed in exact integer / rational arithmetic, so that the inputs
carry the crystal symmetry exactly.

Conventions (shared by every consumer of the generated inputs):
  * real-space lattice L = [a1 a2 a3] (columns, bohr); fractional position x,
    Cartesian r = L x;
  * reciprocal lattice B = 2 pi L^{-T}; a wave vector in reciprocal
    fractional coordinates y has Cartesian value B y;
  * a symmetry operation is {R | t}: x -> R x + t with R an integer matrix in
    lattice coordinates and t fractional; it maps y -> R^{-T} y (Eq. sk of
    the paper with alpha = 0);
  * Gamma-centred mesh n1 x n2 x n3: f = (i/n1, j/n2, l/n3), index
    k = (i*n2 + j)*n3 + l.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass
from fractions import Fraction as Fr
from functools import reduce

import numpy as np


def _lcm(a: int, b: int) -> int:
    return a * b // math.gcd(a, b)


def _fr_inv3(m):
    """Inverse of a 3x3 matrix of Fractions (cofactor formula)."""
    a = [[Fr(x) for x in row] for row in m]
    det = (a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
           - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
           + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]))
    cof = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            r = [x for x in range(3) if x != i]
            c = [x for x in range(3) if x != j]
            minor = a[r[0]][c[0]] * a[r[1]][c[1]] - a[r[0]][c[1]] * a[r[1]][c[0]]
            cof[i][j] = minor * (1 if (i + j) % 2 == 0 else -1)
    return [[cof[j][i] / det for j in range(3)] for i in range(3)], det


def int_inv3(r: np.ndarray) -> np.ndarray:
    """Inverse of a unimodular integer 3x3 matrix, exactly."""
    inv, det = _fr_inv3(r.tolist())
    assert abs(det) == 1, "symmetry matrix is not unimodular"
    out = np.array([[int(x) for x in row] for row in inv], dtype=np.int64)
    assert np.array_equal(out @ r, np.eye(3, dtype=np.int64))
    return out


@dataclass(frozen=True)
class Crystal:
    """A crystal: Bravais lattice kind, lattice constant(s) and atom basis."""
    name: str
    kind: str                 # "fcc" or "hex"
    a: float                  # bohr
    c_over_a: Fr | None       # hex only (exact rational)
    atoms: tuple              # ((species, (Fr, Fr, Fr)), ...) fractional
    weights: tuple            # ((species, weight), ...) for the structure factor

    # -- lattice ---------------------------------------------------------
    def lattice(self) -> np.ndarray:
        a = self.a
        if self.kind == "fcc":
            return 0.5 * a * np.array([[0.0, 1.0, 1.0],
                                       [1.0, 0.0, 1.0],
                                       [1.0, 1.0, 0.0]]).T
        if self.kind == "hex":
            c = a * float(self.c_over_a)
            return np.array([[a, 0.0, 0.0],
                             [-0.5 * a, 0.5 * math.sqrt(3.0) * a, 0.0],
                             [0.0, 0.0, c]]).T
        raise ValueError(self.kind)

    def metric_over_a2(self):
        """g / a^2 with g = L^T L, as exact Fractions."""
        if self.kind == "fcc":
            return [[Fr(1, 2), Fr(1, 4), Fr(1, 4)],
                    [Fr(1, 4), Fr(1, 2), Fr(1, 4)],
                    [Fr(1, 4), Fr(1, 4), Fr(1, 2)]]
        ca2 = self.c_over_a * self.c_over_a
        return [[Fr(1), Fr(-1, 2), Fr(0)],
                [Fr(-1, 2), Fr(1), Fr(0)],
                [Fr(0), Fr(0), ca2]]

    def metric_int(self) -> np.ndarray:
        """An integer multiple of g (for exact tests of R^T g R = g)."""
        g = self.metric_over_a2()
        den = reduce(_lcm, [x.denominator for row in g for x in row], 1)
        return np.array([[int(x * den) for x in row] for row in g], dtype=np.int64)

    def recip_metric_int(self):
        """(M, den): B^T B = (2 pi / a)^2 * M / den with M integer."""
        inv, _ = _fr_inv3(self.metric_over_a2())
        den = reduce(_lcm, [x.denominator for row in inv for x in row], 1)
        m = np.array([[int(x * den) for x in row] for row in inv], dtype=np.int64)
        return m, den

    def volume(self) -> float:
        return abs(float(np.linalg.det(self.lattice())))

    def recip(self) -> np.ndarray:
        return 2.0 * math.pi * np.linalg.inv(self.lattice()).T

    def weight_of(self, species: str) -> float:
        return dict(self.weights)[species]


def si_diamond(a: float = 10.26) -> Crystal:
    """Diamond structure (space group Fd-3m, origin on an atom)."""
    return Crystal("Si", "fcc", a, None,
                   (("Si", (Fr(0), Fr(0), Fr(0))),
                    ("Si", (Fr(1, 4), Fr(1, 4), Fr(1, 4)))),
                   (("Si", 1.0),))


def lif_rocksalt(a: float = 7.6) -> Crystal:
    """Rocksalt structure (Fm-3m)."""
    return Crystal("LiF", "fcc", a, None,
                   (("Li", (Fr(0), Fr(0), Fr(0))),
                    ("F", (Fr(1, 2), Fr(1, 2), Fr(1, 2)))),
                   (("Li", 3.0), ("F", 9.0)))


def mos2_2h(a: float = 5.97, c_over_a: Fr = Fr(39, 10), z: Fr = Fr(623, 1000)) -> Crystal:
    """2H stacking (P6_3/mmc, origin on an inversion centre); z is the
    internal parameter of the chalcogen positions."""
    t, s = Fr(1, 3), Fr(2, 3)
    return Crystal("MoS2", "hex", a, c_over_a,
                   (("Mo", (t, s, Fr(1, 4))), ("Mo", (s, t, Fr(3, 4))),
                    ("S", (t, s, z)), ("S", (s, t, (z + Fr(1, 2)) % 1)),
                    ("S", (s, t, (-z) % 1)), ("S", (t, s, (Fr(1, 2) - z) % 1))),
                   (("Mo", 42.0), ("S", 16.0)))


# ---------------------------------------------------------------------------
# space group
# ---------------------------------------------------------------------------

def _maps_atoms(crys: Crystal, r: np.ndarray, t) -> bool:
    pos = {}
    for sp, x in crys.atoms:
        pos.setdefault(sp, set()).add(tuple(xi % 1 for xi in x))
    for sp, x in crys.atoms:
        y = tuple((sum(int(r[i, j]) * x[j] for j in range(3)) + t[i]) % 1 for i in range(3))
        if y not in pos[sp]:
            return False
    return True


def space_group(crys: Crystal):
    """All operations {R|t} of the crystal, R from the lattice point group.

    Returns (rot int64 [n,3,3], tau list of Fraction triples), ordered by the
    flattened R (lexicographic).  t is reduced to [0,1).
    """
    gi = crys.metric_int()
    rots = []
    for e in itertools.product((-1, 0, 1), repeat=9):
        r = np.array(e, dtype=np.int64).reshape(3, 3)
        if np.array_equal(r.T @ gi @ r, gi):
            rots.append(r)
    rots.sort(key=lambda m: tuple(m.ravel()))
    sp0, x0 = crys.atoms[0]
    cands = [x for sp, x in crys.atoms if sp == sp0]
    out_r, out_t = [], []
    for r in rots:
        rx0 = [sum(int(r[i, j]) * x0[j] for j in range(3)) for i in range(3)]
        for xc in cands:
            t = tuple((xc[i] - rx0[i]) % 1 for i in range(3))
            if _maps_atoms(crys, r, t):
                out_r.append(r)
                out_t.append(t)
                break
    return np.array(out_r, dtype=np.int64), out_t


# ---------------------------------------------------------------------------
# mesh and coset spheres
# ---------------------------------------------------------------------------

class Mesh:
    """Gamma-centred k mesh with exact rotation of mesh points."""

    def __init__(self, n):
        self.n = tuple(int(x) for x in n)
        self.N = reduce(_lcm, self.n, 1)
        idx = np.array(list(itertools.product(range(self.n[0]), range(self.n[1]),
                                              range(self.n[2]))), dtype=np.int64)
        self.idx = idx                                   # [Nk,3]
        self.X = idx * (self.N // np.array(self.n))      # N * f, integer
        self.nk = len(idx)

    def index(self, i, j, l) -> int:
        n1, n2, n3 = self.n
        return ((i % n1) * n2 + (j % n2)) * n3 + (l % n3)

    def f(self, k: int) -> np.ndarray:
        return self.idx[k] / np.array(self.n, dtype=float)

    def rotate(self, rk: np.ndarray, k: int):
        """Mesh index of R^{-T} f_k and the fold G = R^{-T} f_k - f_k'."""
        Xp = rk @ self.X[k]
        step = self.N // np.array(self.n)
        assert np.all(Xp % step == 0), "mesh not invariant under the operation"
        j = Xp // step
        k2 = self.index(*j)
        fold = (Xp - self.X[k2])
        assert np.all(fold % self.N == 0)
        return k2, fold // self.N


def coset_sphere(crys: Crystal, mesh: Mesh, k: int, rho: Fr) -> np.ndarray:
    """Integer vectors m with |B (f_k + m)| <= rho * 2 pi / a, inclusive.

    Exact test: with X = N (f_k + m), |p|^2 = (2pi/a)^2 X^T M X / (den N^2).
    Order: by |p|^2, then m lexicographically.
    """
    M, den = crys.recip_metric_int()
    lat = crys.lattice()
    half = [int(math.ceil(float(rho) * np.linalg.norm(lat[:, i]) / crys.a)) + 1 for i in range(3)]
    rng = [np.arange(-h - 1, h + 2) for h in half]
    m = np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3).astype(np.int64)
    X = m * mesh.N + mesh.X[k]
    val = np.einsum("ni,ij,nj->n", X, M, X)
    lim = rho.numerator ** 2 * den * mesh.N ** 2
    keep = val * rho.denominator ** 2 <= lim
    m, val = m[keep], val[keep]
    # the search box must strictly contain the sphere
    assert np.all(np.abs(m) < np.array(half) + 1)
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], val))
    return m[order]


def norm2_cart(crys: Crystal, mesh: Mesh, X: np.ndarray) -> np.ndarray:
    """|p|^2 in bohr^-2 for integer X = N * (reciprocal fractional vector)."""
    M, den = crys.recip_metric_int()
    val = np.einsum("...i,ij,...j->...", X, M, X).astype(np.float64)
    return (2.0 * math.pi / crys.a) ** 2 * val / (den * mesh.N ** 2)
