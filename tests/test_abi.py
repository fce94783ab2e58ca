"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/css.h (no GPU)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "css.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(css_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2404_19751_gb300 import build
    return build.build()


def test_header_declares_the_hot_path():
    names = _declared()
    for n in ("css_mesh_upload", "css_particles_set", "css_geodesic_neighbors", "css_compute_forces",
              "css_integrate_step", "css_batch_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(css_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_reports_no_device(lib_path):
    from paper_2404_19751_gb300 import _lib
    L = _lib.load(lib_path)
    for n in _lib.SYMBOLS:
        assert hasattr(L, n)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        h = ctypes.c_void_p()
        assert L.css_create(ctypes.byref(h), 0, None) == -8
