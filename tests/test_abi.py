"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/bz.h declares; argument checks answer before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_04457_gb300 import build as B
    B.build()
    from paper_1912_04457_gb300 import bz
    return bz.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(bz_\w+)\s*\(", text, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("bz_init_grid", "bz_set_species", "bz_collision_term", "bz_drift", "bz_step",
                     "bz_moments"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    from paper_1912_04457_gb300 import bz
    assert declared_symbols() <= set(bz.SIGNATURES)


def test_invalid_grid_is_rejected_without_device_work(lib):
    from paper_1912_04457_gb300 import bz
    g = bz.BzGrid()
    g.nx[:] = [1, 1, 1]
    g.np[:] = [0, 4, 4]
    g.dx, g.L = 1.0, 2.0
    h = C.c_void_p()
    assert lib.bz_init_grid(C.byref(h), C.byref(g)) == bz.BZ_EINVAL
    assert b"positive" in lib.bz_last_error(None)
    g.np[:] = [4, 4, 4]
    g.L = -1.0
    assert lib.bz_init_grid(C.byref(h), C.byref(g)) == bz.BZ_EINVAL
    g.L = 2.0
    g.np[:] = [512, 4, 4]
    assert lib.bz_init_grid(C.byref(h), C.byref(g)) == bz.BZ_EINVAL
    assert lib.bz_destroy(None) == bz.BZ_EINVAL
    assert lib.bz_version().startswith(b"libbz")


def test_no_device_reports_enodev(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1912_04457_gb300 import bz
    g = bz.BzGrid()
    g.nx[:] = [1, 1, 1]
    g.np[:] = [4, 4, 4]
    g.dx, g.L = 1.0, 2.0
    h = C.c_void_p()
    assert lib.bz_init_grid(C.byref(h), C.byref(g)) == bz.BZ_ENODEV
    with pytest.raises(bz.BzError):
        bz.Handle(np_=(4, 4, 4))


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_1912_04457_gb300 import bz
    saved = bz._lib
    try:
        bz._lib = None
        with pytest.raises(ImportError):
            bz.load(str(tmp_path / "missing.so"))
    finally:
        bz._lib = saved
