"""The C-ABI library loads and exports every symbol include/lj.h declares;
host-only entry points work without a GPU.  No compute calls here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(lj_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_0709_3225_gb300 import _build, lj
    _build.build()
    return lj.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lj_create", "lj_destroy", "lj_bin", "lj_get_cells", "lj_forces", "lj_step",
                 "lj_energy", "lj_step_host", "lj_check", "lj_grid", "lj_strerror", "lj_version"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_0709_3225_gb300 import lj
    assert set(lj._SIGS) == _declared()


def test_host_only_calls(lib):
    from paper_0709_3225_gb300 import lj
    hdr = open(os.path.join(ROOT, "include", "lj.h")).read()
    ver = int(re.search(r"#define LJ_ABI_VERSION (\d+)", hdr).group(1))
    assert lj.lj_version() == ver
    for code in range(8):
        assert lj.lj_strerror(code) and "unknown" not in lj.lj_strerror(code)
    assert "unknown" in lj.lj_strerror(99)
    # Section 3.2 worked example: L = 11, rc = 2.5 -> 4 cells per side.
    assert lj.lj_grid(lj.make_params(100, 11.0, rc=2.5)) == 4
    # Sizes of the named workloads.
    from paper_0709_3225_gb300 import inputs
    for name, nc in (("fluid-2k", 5), ("fluid-131k", 21), ("fluid-4m", 67), ("fm-32k", 13)):
        w = inputs.WORKLOADS[name]
        assert lj.lj_grid(lj.make_params(w.n, w.box)) == nc


def test_grid_agrees_with_oracle(lib, oracle_mod):
    from paper_0709_3225_gb300 import lj
    for L in (7.5, 7.6, 8.4, 11.0, 13.43677, 53.74708, 167.95962, 321.0):
        assert lj.lj_grid(lj.make_params(10, L)) == oracle_mod.ncells(L, 2.5)
        # subdivision k = 2: n = floor(2L / rc) >= 5 half-size cells per side
        assert lj.lj_grid(lj.make_params(10, L, cell_subdiv=2)) == oracle_mod.ncells(L, 2.5, k=2)
    assert lj.lj_grid(lj.make_params(10, 6.25, cell_subdiv=2)) == 5
    with pytest.raises(lj.LJError):
        lj.lj_grid(lj.make_params(10, 6.2, cell_subdiv=2))      # 4 cells < 2k + 1


@pytest.mark.parametrize("field,value,code", [
    ("box", 7.4, 2), ("box", 0.0, 1), ("box", float("nan"), 1), ("sigma", 0.0, 1), ("rc", -1.0, 1),
    ("mass", 0.0, 1), ("eps", -1.0, 1), ("shift_mode", 3, 1), ("precision", 2, 1),
    ("cell_subdiv", 3, 1), ("cell_subdiv", -1, 1), ("flags", 8, 1), ("flags", 3, 1), ("n", -1, 1), ("n", 2 ** 31, 6), ("box", 1e6, 6),
])
def test_bad_parameters_rejected(lib, field, value, code):
    from paper_0709_3225_gb300 import lj
    p = lj.make_params(1000, 20.0)
    setattr(p, field, value)
    nc = ctypes.c_int32()
    assert lib.lj_grid(ctypes.byref(p), ctypes.byref(nc)) == code
    # lj_create validates before touching the GPU.
    h = ctypes.c_void_p()
    assert lib.lj_create(ctypes.byref(h), ctypes.byref(p), None) == code
    assert not h.value


@pytest.mark.parametrize("precision,flags", [("fp64", 0), ("mixed", 1), ("mixed", 2)])
def test_subdivision_two_needs_the_warp_kernel(lib, precision, flags):
    from paper_0709_3225_gb300 import lj
    p = lj.make_params(1000, 20.0, precision=precision, cell_subdiv=2, flags=flags)
    nc = ctypes.c_int32()
    assert lib.lj_grid(ctypes.byref(p), ctypes.byref(nc)) == 1


def test_null_arguments_rejected(lib):
    assert lib.lj_bin(None, None) == 1
    assert lib.lj_forces(None, None, None, None, None) == 1
    assert lib.lj_step(None, None, None, None, 1) == 1
    assert lib.lj_check(None) == 1
    assert lib.lj_grid(None, None) == 1
    assert lib.lj_create(None, None, None) == 1
    lib.lj_destroy(None)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_0709_3225_gb300 import lj
    monkeypatch.setattr(lj, "_lib", None)
    monkeypatch.setattr(lj, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lj.load()
