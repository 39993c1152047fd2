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


def test_host_side_argument_checks_without_a_gpu():
    """Descriptions and arguments the library rejects before any CUDA call:
    CF_EINVAL with the reason in cf_last_error()."""
    import ctypes as C
    from paper_2007_15405_gb300 import capfilm as cf
    L = cf.load_library()

    def desc(nx=16, ny=12, nz=20, tau=(1.0, 1.0), precision=0, flags=0):
        return cf.LatticeDesc(nx, ny, nz, 1, (C.c_double * 2)(*tau), 3.6, 10.0, 1.5, 1.5, precision,
                              None, None, flags)

    cases = [(desc(nx=2), "dimensions"), (desc(nz=0), "dimensions"),
             (desc(nx=512, ny=512, nz=256), "too large"), (desc(tau=(0.5, 1.0)), "tau"),
             (desc(tau=(1.0, float("nan"))), "tau"), (desc(precision=7), "precision"),
             (desc(flags=32), "unknown flag"), (desc(flags=16 | 1), "CF_INERTIAL")]
    for d, why in cases:
        h = C.c_void_p()
        rc = L.cf_create(C.byref(d), C.byref(h))
        assert cf.STATUS_NAMES[rc] == "CF_EINVAL", why
        assert why in L.cf_last_error().decode()
    assert cf.STATUS_NAMES[L.cf_create(None, None)] == "CF_EINVAL"
    for call in (lambda: L.cf_step(None, C.c_longlong(1)), lambda: L.cf_sync(None),
                 lambda: L.cf_save(None, b"x"), lambda: L.cf_load(None, b"x"),
                 lambda: L.cf_remove_mass(None, C.c_double(1.0)),
                 lambda: L.cf_batch_step(None, C.c_longlong(1))):
        assert cf.STATUS_NAMES[call()] == "CF_EINVAL"
    assert cf.STATUS_NAMES[L.cf_destroy(None)] == "CF_OK"  # like free(NULL)
