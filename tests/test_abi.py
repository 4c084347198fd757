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
