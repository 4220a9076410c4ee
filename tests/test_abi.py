"""The C-ABI library builds, loads and exports every symbol include/fkp.h
declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re
import subprocess

import numpy as np
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


def test_binding_constants_match_the_header():
    """Every FKP_* enum value of include/fkp.h (output flags, contraction
    modes, error codes) has the same value in the Python binding."""
    src = open(os.path.join(ROOT, "include", "fkp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", src):
        for name, val in re.findall(r"\b(FKP_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            consts[name] = int(val)
    assert "FKP_XHAT_OBJECT" in consts and "FKP_CONTRACT_BF16X6" in consts
    for name, val in consts.items():
        if hasattr(fkp, name):
            assert getattr(fkp, name) == val, name
        elif name != "FKP_OK":
            assert fkp.ERRORS.get(val) == name, name


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


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structs have the sizes the C compiler gives the
    header's structs on this machine."""
    assert ctypes.sizeof(fkp.Catalog) == 5 * 8 + 8 + 8
    assert ctypes.sizeof(fkp.PBins) == 24
    assert ctypes.sizeof(fkp.BShells) == 16
    names = {"fkp_catalog_t": fkp.Catalog, "fkp_geometry_t": fkp.Geometry, "fkp_pbins_t": fkp.PBins,
             "fkp_bshells_t": fkp.BShells, "fkp_power_out": fkp.PowerOut, "fkp_bisp_out": fkp.BispOut,
             "fkp_request_t": fkp.Request, "fkp_server_stats_t": fkp.ServerStats}
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include "fkp.h"\nint main(void) {\n' +
                   "".join(f'  printf("%zu\\n", sizeof({n}));\n' for n in names) + "  return 0;\n}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    for (n, cls), size in zip(names.items(), sizes):
        assert ctypes.sizeof(cls) == size, n


class _FakeCudaTensor:
    """Stands in for a CUDA tensor on a machine without a GPU: only what the
    binding's argument checks look at."""
    is_cuda = True

    def __init__(self, dtype, n, index=0):
        import torch
        self.dtype, self._n, self.device = dtype, n, torch.device("cuda", index)

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n

    def data_ptr(self):
        raise AssertionError("the binding must reject this field before reading its pointer")


def test_binding_rejects_bad_fields_before_any_launch():
    """A field of the wrong dtype, size or device is refused in Python, before
    the C call (which would read N^3 float32 values from its pointer)."""
    torch = pytest.importorskip("torch")
    import paper_1506_02729_gb300 as fkp
    N = 16
    fkp.check_field(_FakeCudaTensor(torch.float32, N ** 3), N, 0)
    with pytest.raises(TypeError):
        fkp.check_field(_FakeCudaTensor(torch.float16, N ** 3), N, 0)
    with pytest.raises(TypeError):
        fkp.check_field(_FakeCudaTensor(torch.float64, N ** 3), N, 0)
    with pytest.raises(ValueError):
        fkp.check_field(_FakeCudaTensor(torch.float32, N ** 3 - 1), N, 0)
    with pytest.raises(ValueError):
        fkp.check_field(_FakeCudaTensor(torch.float32, N ** 3, index=1), N, 0)
    with pytest.raises(TypeError):
        fkp.check_field(np.zeros((N, N, N), np.float32), N, 0)
