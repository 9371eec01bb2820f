"""Pins of the oracle's symmetry tables against group theory (Sec. III.C)."""
import itertools
import math
import os

import numpy as np
import pytest

from conftest import oracle_case
from oracle.tables import Group, MeshTables

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("name,order", [("si2", 48), ("lif4", 48), ("mos2_331", 24)])
def test_group_order_and_closure(name, order):
    d, inp, grp, mt, b = oracle_case(name)
    assert grp.n == order
    # every product and inverse is in the set (checked in Group), identity present
    assert np.array_equal(grp.rot[grp.identity], np.eye(3, dtype=np.int64))
    # Cartesian matrices are orthogonal
    for a in grp.cart:
        assert np.allclose(a @ a.T, np.eye(3), atol=1e-12)


def _burnside_star_count(rot, mesh):
    """Number of orbits of the mesh = average number of fixed points (orbit-
    counting lemma), with fixed points found by brute force."""
    n = np.array(mesh, dtype=float)
    f = np.array(list(itertools.product(*[range(x) for x in mesh]))) / n
    tot = 0
    for r in rot:
        rk = np.linalg.inv(r).T
        d = f @ rk.T - f
        tot += int(np.sum(np.all(np.abs(d - np.round(d)) < 1e-9, axis=1)))
    assert tot % len(rot) == 0
    return tot // len(rot)


@pytest.mark.parametrize("mesh", [(2, 2, 2), (4, 4, 4), (8, 8, 8), (12, 12, 12)])
def test_star_count_fcc(mesh):
    d, inp, grp, mt, b = oracle_case("si2")
    m = MeshTables(grp, mesh)
    assert len(m.star_rep) == _burnside_star_count(grp.rot, mesh)
    sizes = np.array([len(s) for s in m.stars])
    assert sizes.sum() == np.prod(mesh)
    # orbit-stabiliser: |star| * |little group| = |S|
    for a, p in enumerate(m.star_rep):
        assert sizes[a] * len(m.little_group(p)) == grp.n
    # representative is the lowest index, s_k maps it onto k
    for k in range(m.nk):
        a = m.star_of[k]
        assert m.star_rep[a] == min(m.stars[a])
        assert m.rotk[m.s_k[k], m.star_rep[a]] == k


def test_star_count_values():
    """Irreducible point counts of Gamma-centred fcc meshes under Oh."""
    d, inp, grp, mt, b = oracle_case("si2")
    got = [len(MeshTables(grp, (n, n, n)).star_rep) for n in (4, 8, 12)]
    assert got == [8, 29, 72]


def _class_key(grp, cls):
    out = {}
    for c in set(cls.tolist()):
        s = int(np.nonzero(cls == c)[0][0])
        a = grp.cart[s]
        order = 1
        m = a.copy()
        while not np.allclose(m, np.eye(3), atol=1e-9):
            m = m @ a
            order += 1
        out[c] = (int(round(np.linalg.det(a))), int(round(np.trace(a))), order,
                  int(np.sum(cls == c)))
    return out


def test_characters_oh_textbook():
    d, inp, grp, mt, b = oracle_case("si2")
    chi, dims, cls = grp.characters()
    keys = _class_key(grp, cls)
    lines = [l.split() for l in open(os.path.join(GOLDEN, "oh_character_table.txt"))
             if l.strip() and not l.startswith("#")]
    colkeys = [tuple(int(x) for x in k.split(",")) for k in lines[0][1:]]
    table = {l[0]: [int(x) for x in l[1:]] for l in lines[1:]}
    assert len(set(keys.values())) == len(keys) == 10
    ours = set()
    for mu in range(len(dims)):
        row = []
        for ck in colkeys:
            c = [c for c, k in keys.items() if k == ck][0]
            row.append(int(chi[mu][np.nonzero(cls == c)[0][0]]))
        ours.add(tuple(row))
    assert ours == {tuple(v) for v in table.values()}
    # the bright irrep of Oh is T1u
    t1u = tuple(table["T1u"])
    assert [mu for mu in range(len(dims)) if tuple(
        int(chi[mu][np.nonzero(cls == [c for c, k in keys.items() if k == ck][0])[0][0]])
        for ck in colkeys) == t1u] == b.bright()


@pytest.mark.parametrize("name", ["si2", "mos2_331"])
def test_character_orthogonality(name):
    d, inp, grp, mt, b = oracle_case(name)
    chi, dims, cls = grp.characters()
    n = grp.n
    assert len(dims) == len(set(cls.tolist()))                 # #irreps = #classes
    assert int(np.sum(dims ** 2)) == n                         # |S| = sum d^2
    assert np.array_equal(chi @ chi.T, n * np.eye(len(dims), dtype=np.int64))   # Eq. LOT
    assert np.array_equal(chi[:, grp.identity], dims)


def test_d6h_bright_irreps():
    """In D6h the polar vector splits into E1u (in plane) + A2u (along z)."""
    d, inp, grp, mt, b = oracle_case("mos2_331")
    chi, dims, cls = grp.characters()
    br = b.bright()
    assert sorted(dims[br].tolist()) == [1, 2]
    axz = np.array([round(a[2, 2]) for a in grp.cart])
    inplane = np.array([round(np.trace(a) - a[2, 2]) for a in grp.cart])
    rows = {tuple(chi[mu]) for mu in br}
    assert rows == {tuple(axz), tuple(inplane)}
