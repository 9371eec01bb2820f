"""The C ABI library loads and exports every function declared in include/*.h
(no compute calls: these run without a GPU)."""
import glob
import os
import re

import pytest

from paper_2603_24860_gb300 import bse

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bse_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def library():
    if not os.path.exists(bse.LIB_PATH):
        from paper_2603_24860_gb300.build import build
        build()
    return bse.lib()


def test_every_declared_symbol_is_exported(library):
    names = _declared()
    assert {"bse_create", "bse_build_block", "bse_block_spectrum", "bse_pairdens"} <= names
    for n in names:
        assert hasattr(library, n), n


def test_binding_covers_the_header(library):
    assert _declared() == set(bse.EXPORTS)


def test_last_error_empty_string(library):
    assert isinstance(library.bse_last_error(), bytes)


def test_binding_has_no_fallback(monkeypatch, tmp_path):
    """Without the compiled library the binding raises instead of computing."""
    monkeypatch.setattr(bse, "_lib", None)
    monkeypatch.setattr(bse, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        bse.lib()
