"""The C-ABI library builds, loads and exports every entry point include/nnp.h
declares (no GPU needed: nothing here calls a compute entry point)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "nnp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nnp_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2207_14276_gb300 import build
    return build.build()


def test_header_declares_boundary(libpath):
    syms = declared_symbols()
    for s in ("nnp_create", "nnp_energy_forces", "nnp_energy_forces_batch", "nnp_destroy",
              "nnp_last_error", "nnp_sync_status", "nnp_energy_forces_host"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nnp_[a-z_0-9]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_python_binding_matches_header(libpath):
    import paper_2207_14276_gb300 as pkg
    assert sorted(pkg.EXPORTS) == declared_symbols()
    L = ctypes.CDLL(libpath)
    for s in declared_symbols():
        assert hasattr(L, s)


def test_last_error_is_empty_string_initially(libpath):
    L = ctypes.CDLL(libpath)
    L.nnp_last_error.restype = ctypes.c_char_p
    assert L.nnp_last_error() == b""


def test_bounds_checked_build_exports_the_same_symbols(libpath):
    """libnnp_debug.so (the sources built with -DNNP_DEBUG_BOUNDS) has the same
    entry points; nnp_build_flags tells the two builds apart."""
    from paper_2207_14276_gb300 import build
    dbg = build.LIB_DEBUG
    assert os.path.exists(dbg)
    out = subprocess.run(["nm", "-D", "--defined-only", dbg], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nnp_[a-z_0-9]+)", out))
    assert [s for s in declared_symbols() if s not in exported] == []
    rel, deb = ctypes.CDLL(libpath), ctypes.CDLL(dbg)
    assert rel.nnp_build_flags() == 0
    assert deb.nnp_build_flags() == 1   # NNP_BUILD_BOUNDS_CHECKS


def test_index_check_bookkeeping(libpath):
    """The check the bounds-checked kernels run, executed on the host: in range
    leaves the status alone; out of range ORs 32 into status[0] and keeps the
    first failing site in status[3]; bad arguments return -1."""
    L = ctypes.CDLL(libpath)
    L.nnp_debug_check_index.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int)]
    st = (ctypes.c_int * 4)(0, 0, 0, 0)
    for i, n in ((0, 1), (5, 6), (2 ** 40, 2 ** 40 + 1)):
        assert L.nnp_debug_check_index(3, i, n, st) == 1
    assert list(st) == [0, 0, 0, 0]
    st = (ctypes.c_int * 4)(4, 7, 9, 0)          # other flags and counts stay
    assert L.nnp_debug_check_index(6, 10, 10, st) == 0
    assert list(st) == [4 | 32, 7, 9, 6]
    assert L.nnp_debug_check_index(2, -1, 10, st) == 0
    assert L.nnp_debug_check_index(9, 2 ** 33, 2 ** 32, st) == 0
    assert list(st) == [4 | 32, 7, 9, 6]         # the first site is kept
    assert L.nnp_debug_check_index(0, 0, 1, st) == -1
    assert L.nnp_debug_check_index(11, 0, 1, st) == -1
    assert L.nnp_debug_check_index(1, 0, 1, None) == -1
