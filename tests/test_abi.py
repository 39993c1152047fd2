"""The C ABI library loads and exports every entry point include/capfilm.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "capfilm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(cf_[a-z0-9_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_15405_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = declared_symbols()
    assert "cf_step" in syms and "cf_create" in syms and len(syms) >= 15


def test_library_exports_all_declared_symbols(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2007_15405_gb300 import capfilm
    assert sorted(capfilm.exported_symbols()) == declared_symbols()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2007_15405_gb300 import capfilm
    saved = capfilm._lib
    capfilm._lib = None
    try:
        with pytest.raises(capfilm.CapfilmError):
            capfilm.load_library(str(tmp_path / "nope.so"))
    finally:
        capfilm._lib = saved


def test_oracle_library_is_separate():
    """The oracle is a different shared object sharing no symbols with the
    CUDA library."""
    import oracle
    L = oracle.lib()
    assert not hasattr(L, "cf_step")
    src = open(os.path.join(ROOT, "oracle", "capfilm_oracle.c")).read()
    assert "capfilm.h" not in src and "cf_common" not in src
