"""Shared fixtures.  Tests marked ``gpu`` need a CUDA device and the built
library; everything else runs on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled library")


_CASES = {}


def oracle_case(name):
    """(inputs dict, Inputs, Group, MeshTables, Basis) of a configuration, cached."""
    if name not in _CASES:
        from synth import generate
        from oracle.hamiltonian import Inputs
        from oracle.projection import Basis
        from oracle.tables import Group, MeshTables
        d = generate(name)
        inp = Inputs(d)
        grp = Group(d["rot"], d["tau"], d["lattice"])
        mt = MeshTables(grp, d["mesh"])
        _CASES[name] = (d, inp, grp, mt, Basis(inp, grp, mt))
    return _CASES[name]


_H = {}


def oracle_h(name, terms="dxw"):
    """Full oracle Hamiltonian of a small configuration, cached."""
    key = (name, terms)
    if key not in _H:
        from oracle.hamiltonian import full_hamiltonian, head_correction
        d, inp, grp, mt, b = oracle_case(name)
        if (name, "wdiv") not in _H:
            _H[(name, "wdiv")] = head_correction(inp)
        wd = _H[(name, "wdiv")]
        _H[key] = full_hamiltonian(inp, mt, w_div=wd, terms=terms)
    return _H[key]
