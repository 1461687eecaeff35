"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/dg.h declares (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1812_04789_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    return sorted(set(re.findall(r"^dg_status\s+(dg_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    assert os.path.exists(path)
    return ctypes.CDLL(path)


def test_header_declares_the_abi():
    names = declared_symbols()
    for n in ["dg_mesh_create", "dg_residual", "dg_jvp", "dg_pmg_setup", "dg_pmg_apply",
              "dg_fgmres_step"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == declared_symbols()


def test_library_is_sm103a_and_dynamic_symbols():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for name in declared_symbols():
        assert re.search(r"\bT %s\b" % name, out), name
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_loads_and_rejects_null_handles(lib):
    L = binding.load()
    # argument validation happens before any CUDA call
    assert L.dg_mesh_destroy(None) == 1
    assert L.dg_residual(None, None, None, None, None) == 1
    assert L.dg_pmg_apply(None, None, None, None) == 1
    out = ctypes.c_void_p()
    d = binding.MeshDesc()
    d.dim = 4
    ph = binding.PhysicsDesc(1.4, 0.72, 0.0, 1.0, 0.0, 0.1)
    assert L.dg_mesh_create(ctypes.byref(d), ctypes.byref(ph), None, ctypes.byref(out)) == 1
    assert out.value is None
