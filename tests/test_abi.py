"""CPU-side checks of the C ABI: liblagp.so builds, loads and exports every
function include/lagp.h declares; argument errors are reported without any
GPU work.  (Compute calls need a GPU and live in the -m gpu tests.)"""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lagp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lagp_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1310_5182_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("lagp_knn", "lagp_alc_select", "lagp_predict", "lagp_mle_step", "lagp_create",
              "lagp_destroy", "lagp_last_error", "lagp_agp", "lagp_predict_grad"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    _, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (lagp_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_status_strings_and_null_context(lib):
    L, _ = lib
    L.lagp_status_string.restype = ctypes.c_char_p
    assert L.lagp_status_string(0) == b"LAGP_OK"
    assert L.lagp_status_string(2) == b"LAGP_ENOTPD"
    P = ctypes.c_void_p
    # a NULL context is rejected before any CUDA call
    L.lagp_knn.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, P, ctypes.c_int64,
                           P, ctypes.c_int32, P, P]
    assert L.lagp_knn(None, None, 10, 2, 0, None, 1, None, 5, None, None) == 1
    assert L.lagp_destroy(None) == 0
    L.lagp_create.argtypes = [P, ctypes.c_int, P]
    assert L.lagp_create(None, 0, None) == 1


def test_binding_refuses_to_import_without_library(tmp_path):
    # the binding raises instead of falling back when liblagp.so is absent
    import importlib.util
    src = os.path.join(ROOT, "paper_1310_5182_gb300", "lagp.py")
    dst = tmp_path / "lagp.py"
    dst.write_text(open(src).read())
    spec = importlib.util.spec_from_file_location("lagp_copy", dst)
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
