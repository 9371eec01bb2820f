"""The library's host tables (csrc/host_tables.cpp: space group, rotated k
mesh, stars and s_k, classes and characters by Burnside-Dixon, multiplets
and product-basis orbits), built on the CPU by a small C++ driver and
compared bit for bit with the oracle (Sec. III.C.1-4).  No GPU: the same
host code runs inside bse_create."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.tables import Group, MeshTables, orbits
from synth import generate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_24860_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.isfile(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("g++ or the CUDA headers are not available")
    exe = str(tmp_path_factory.mktemp("host") / "host_tables_driver")
    cmd = [cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", inc,
           os.path.join(ROOT, "tests", "host_tables_driver.cpp"), os.path.join(CSRC, "host_tables.cpp"),
           "-o", exe, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def _run(driver, d, tmp):
    inp, out = str(tmp / "in.bin"), str(tmp / "out.bin")
    rot = np.ascontiguousarray(d["rot"], dtype=np.int32)
    with open(inp, "wb") as f:
        f.write(np.ascontiguousarray(d["lattice"], dtype=np.float64).tobytes())
        f.write(np.int32(len(rot)).tobytes())
        f.write(rot.tobytes())
        f.write(np.ascontiguousarray(d["tau"], dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(d["mesh"], dtype=np.int32).tobytes())
        f.write(np.int32(d["nv"]).tobytes())
        f.write(np.int32(d["nc"]).tobytes())
        f.write(np.ascontiguousarray(d["eps"], dtype=np.float64).tobytes())
    r = subprocess.run([driver, inp, out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    raw = open(out, "rb").read()
    pos = 0

    def take(dtype, n):
        nonlocal pos
        a = np.frombuffer(raw, dtype=dtype, count=n, offset=pos)
        pos += a.nbytes
        return a
    nk, nops, nstars, nirr = take(np.int32, 4)
    N, norb = take(np.int64, 2)
    t = {"rotk": take(np.int32, nops * nk).reshape(nops, nk), "star_of": take(np.int32, nk),
         "star_rep": take(np.int32, nstars), "s_k": take(np.int32, nk), "class_of": take(np.int32, nops),
         "chi": take(np.int32, nirr * nops).reshape(nirr, nops), "irrep_dim": take(np.int32, nirr),
         "bright": take(np.int32, nirr), "orbit_of": take(np.int32, N), "n_orbits": int(norb)}
    t["fold"] = take(np.int32, nops * nk * 3).reshape(nops, nk, 3)
    assert pos == len(raw)
    return t


@pytest.mark.parametrize("name", ["si2", "si4", "lif4", "mos2_331"])
def test_host_tables_match_the_oracle(driver, tmp_path, name):
    d = generate(name)
    t = _run(driver, d, tmp_path)
    grp = Group(d["rot"], d["tau"], d["lattice"])
    mt = MeshTables(grp, d["mesh"])
    chi, dims, cls = grp.characters()
    assert np.array_equal(t["rotk"], mt.rotk)
    assert np.array_equal(t["fold"], mt.fold)
    assert np.array_equal(t["star_of"], mt.star_of)
    assert np.array_equal(t["star_rep"], mt.star_rep)
    assert np.array_equal(t["s_k"], mt.s_k)
    assert np.array_equal(t["class_of"], cls)
    assert np.array_equal(t["chi"], chi)
    assert np.array_equal(t["irrep_dim"], dims)
    assert np.array_equal(t["bright"], np.rint(chi @ grp.vector_character() / grp.n).astype(int))
    orb = orbits(mt, np.asarray(d["eps"]), int(d["nv"]), int(d["nc"]))
    want = np.zeros(len(t["orbit_of"]), dtype=np.int64)
    for o, mem in enumerate(orb):
        want[mem] = o
    assert t["n_orbits"] == len(orb)
    assert np.array_equal(t["orbit_of"], want)


def _read_bases(path, n_irreps):
    raw = open(path, "rb").read()
    pos = 0

    def take(dtype, n):
        nonlocal pos
        a = np.frombuffer(raw, dtype=dtype, count=int(n), offset=pos)
        pos += a.nbytes
        return a

    def basis():
        dim = int(take(np.int64, 1)[0])
        col_orbit = take(np.int32, dim)
        col_off = take(np.int64, dim + 1)
        coef = take(np.complex128, col_off[-1])
        return col_orbit, col_off, coef
    gam_per_s, norb = take(np.int64, 2)
    orbit_off = take(np.int64, norb + 1)
    members = take(np.int64, orbit_off[-1])
    out = []
    for _ in range(n_irreps):
        whole = basis()
        d = int(take(np.int32, 1)[0])
        out.append((whole, [basis() for _ in range(d)]))
    assert pos == len(raw)
    return int(gam_per_s), orbit_off, members, out


def _dense(b, orbit_off, members, n):
    col_orbit, col_off, coef = b
    U = np.zeros((n, len(col_orbit)), dtype=np.complex128)
    for c, o in enumerate(col_orbit):
        U[members[orbit_off[o]:orbit_off[o + 1]], c] = coef[col_off[c]:col_off[c + 1]]
    return U


@pytest.mark.parametrize("name", ["si2", "si4", "lif4", "mos2_331"])
def test_host_bases_match_the_oracle(driver, tmp_path, name):
    """The orbit-wise bases of every irrep (Eq. projection) and the partner
    bases with their transfers (Sec. III.C.3), built by the library's host
    code from the oracle's band rotations (Eq. Ts), against the oracle's
    canonical U_mu and U_1, U_i."""
    from oracle.hamiltonian import Inputs
    from oracle.projection import Basis, PartnerBasis, band_rotation
    from oracle.tables import multiplets
    d = generate(name)
    inp = Inputs(d)
    grp = Group(d["rot"], d["tau"], d["lattice"])
    mt = MeshTables(grp, d["mesh"])
    nv, nc = int(d["nv"]), int(d["nc"])
    eps = np.asarray(d["eps"])
    gam = []   # the library's layout: per operation, per k the multiplet blocks [target][source]
    for s in range(grp.n):
        for k in range(mt.nk):
            G = band_rotation(inp, grp, mt, s, k)
            for m in list(multiplets(eps[k], 0, nv)) + list(multiplets(eps[k], nv, nv + nc)):
                gam.append(G[np.ix_(m, m)].ravel())
    gam = np.concatenate(gam).astype(np.complex128)
    gpath, bpath = tmp_path / "gamma.bin", tmp_path / "bases.bin"
    gpath.write_bytes(gam.tobytes())
    # the tables (written first) are checked by the test above
    inp_path, out_path = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    _run(driver, d, tmp_path)
    r = subprocess.run([driver, inp_path, out_path, str(gpath), str(bpath)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    b = Basis(inp, grp, mt)
    gps, orbit_off, members, bases = _read_bases(str(bpath), len(b.dims))
    assert gps * grp.n == len(gam)
    for mu, (whole, parts) in enumerate(bases):
        U = _dense(whole, orbit_off, members, inp.N)
        ref, _ = b.basis(mu)
        assert U.shape == ref.shape, (name, mu)
        assert U.size == 0 or np.abs(U - ref).max() <= 1e-10, (name, mu)
        pb = PartnerBasis(b, mu)
        assert len(parts) == len(pb.U), (name, mu)
        for i, p in enumerate(parts):
            Ui = _dense(p, orbit_off, members, inp.N)
            assert Ui.shape == pb.U[i].shape, (name, mu, i)
            assert Ui.size == 0 or np.abs(Ui - pb.U[i]).max() <= 1e-10, (name, mu, i)
