"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU and exports
every function declared in include/grpic.h; the binding covers them all."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(grpic_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_0904_0232_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("grpic_create", "grpic_destroy", "grpic_load_particles", "grpic_step", "grpic_get_fields",
                 "grpic_get_particles", "grpic_set_fields", "grpic_set_uniform_field"):
        assert must in names
    assert len(names) >= 19


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_0904_0232_gb300 import grpic

    assert set(declared_functions()) <= set(grpic.EXPORTS)
    grpic.load_library(lib_path)
    assert grpic.load_library().grpic_status_string(4) == b"GRPIC_ERR_CFL"


def test_config_layout_matches_header(lib_path):
    """Invalid configurations are rejected before any device call (no GPU needed)."""
    from paper_0904_0232_gb300 import grpic

    lib = grpic.load_library(lib_path)
    h = ctypes.c_void_p()
    bad = grpic.grpic_config(4, 16, 16, 1.0, 0.5, 1.0, 0.4, 0, 2, 0.0, 0, 1, 0)  # nx < 8
    assert lib.grpic_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    cfl = grpic.grpic_config(16, 16, 16, 1.0, 0.5, 1.0, 0.6, 0, 2, 0.0, 0, 1, 0)  # c dt >= 1/sqrt(3)
    assert lib.grpic_create(ctypes.byref(cfl), None, ctypes.byref(h)) == 4
    spin = grpic.grpic_config(16, 16, 16, 1.0, 1.5, 1.0, 0.4, 0, 2, 0.0, 0, 1, 0)  # |a| > m
    assert lib.grpic_create(ctypes.byref(spin), None, ctypes.byref(h)) == 1
