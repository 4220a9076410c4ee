"""The C-ABI library builds, loads and exports every symbol include/fkp.h
declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1506_02729_gb300 as fkp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fkp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fkp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1506_02729_gb300 import build
    return build.build()


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(fkp.EXPORTS)


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for s in declared_symbols():
        assert hasattr(L, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    for s in declared_symbols():
        assert re.search(rf"\bT {s}\b", out), s


def test_version_and_error_without_gpu(built):
    assert "sm_103a" in fkp.version()
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = fkp.lib().fkp_context_create(0, 0, ctypes.byref(h))
    assert rc != 0
    assert fkp.lib().fkp_last_error().decode()


def test_moment_tables_reproduce_the_multipole_sums(built):
    """The host tables that turn the trace-reduced moment fields into k_z-power
    groups reproduce S_2 = (k.x^)^2 and S_4 = (k.x^)^4 (no GPU)."""
    fkp.check_tables()


def test_struct_layouts_match_header():
    # sizes the C compiler gives the same structs (x86-64 / aarch64 LP64)
    assert ctypes.sizeof(fkp.Catalog) == 5 * 8 + 8 + 8
    assert ctypes.sizeof(fkp.PBins) == 24
    assert ctypes.sizeof(fkp.BShells) == 16
