"""The C-ABI library loads without a GPU and exports every symbol include/mgc.h
declares; the Python binding declares exactly those symbols."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mgc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mgc_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_00501_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["mgc_lattice_create", "mgc_gauge_create", "mgc_clover_create", "mgc_apply_D",
                 "mgc_apply_Ddag", "mgc_sap_smooth", "mgc_solve", "mgc_force"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_matches_header():
    from paper_2112_00501_gb300 import _lib

    assert sorted(_lib.SIGNATURES) == declared_symbols()


def test_host_side_argument_checks(lib):
    """Shape and argument validation runs on the host, before any CUDA call."""
    from paper_2112_00501_gb300 import _lib

    L = _lib.load()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(8, 8, 8, 8)
    ok_block = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert L.mgc_lattice_create(dims, ok_block, -1, ctypes.byref(h)) == _lib.MGC_OK
    assert L.mgc_lattice_volume(h) == 8 ** 4
    assert L.mgc_spinor_bytes(h, 64, 2) == 2 * 8 ** 4 * 192
    assert L.mgc_spinor_bytes(h, 16, 1) == 8 ** 4 * 52
    L.mgc_lattice_destroy(h)
    # odd number of blocks along x
    bad = (ctypes.c_int * 4)(12, 8, 8, 8)
    assert L.mgc_lattice_create(bad, ok_block, -1, ctypes.byref(h)) == _lib.MGC_ERR_UNSUPPORTED_SHAPE
    # block extent not a power of two
    b3 = (ctypes.c_int * 4)(3, 4, 4, 4)
    assert L.mgc_lattice_create(dims, b3, -1, ctypes.byref(h)) == _lib.MGC_ERR_UNSUPPORTED_SHAPE
    # bad boundary condition
    assert L.mgc_lattice_create(dims, ok_block, 0, ctypes.byref(h)) == _lib.MGC_ERR_INVALID_ARG
    assert b"t_bc" in L.mgc_last_error()
    assert L.mgc_status_string(_lib.MGC_ERR_TIMEOUT) == b"MGC_ERR_TIMEOUT"


def test_product_path_is_independent_of_the_oracle():
    """The package and its CUDA sources neither import, include nor link
    anything under oracle/, and the oracle does not use the package beyond
    the seeded input generators."""
    pkg = os.path.join(ROOT, "paper_2112_00501_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".h")):
                continue
            src = open(os.path.join(dirpath, f)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle\b", src, re.M), f
            assert "liboracle" not in src and "oracle.c" not in src and "oracle.h" not in src, f
    for f in ("oracle.py", "oracle.c", "build.py", "__init__.py"):
        src = open(os.path.join(ROOT, "oracle", f)).read()
        for m in re.finditer(r"paper_2112_00501_gb300\.?(\w*)", src):
            assert m.group(1) in ("", "synth"), (f, m.group(0))
    import subprocess
    lib_path = os.path.join(pkg, "libmgc.so")
    if os.path.exists(lib_path):
        deps = subprocess.run(["ldd", lib_path], capture_output=True, text=True).stdout
        assert "oracle" not in deps
