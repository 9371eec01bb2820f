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
