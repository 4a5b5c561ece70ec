"""The C-ABI library loads and exports every function include/qdvm.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(qdvm_[a-z0-9_]+)\s*\(", src, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def _lib_path():
    import importlib.util

    spec = importlib.util.spec_from_file_location("qdvm_build", os.path.join(ROOT, "paper_1201_3986_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)

    if not b.up_to_date():
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and nvcc unavailable")
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("qdvm_plan_create", "qdvm_eval", "qdvm_eval_batched", "qdvm_vjp", "qdvm_jvp", "qdvm_moments",
                 "qdvm_plan_destroy", "qdvm_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"missing exports: {missing}"


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(_lib_path())
    lib.qdvm_status_string.restype = ctypes.c_char_p
    lib.qdvm_status_string.argtypes = [ctypes.c_int]
    assert lib.qdvm_status_string(0) == b"ok"
    assert lib.qdvm_status_string(6) == b"bad plan handle"
    lib.qdvm_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.qdvm_version()
    # argument validation happens before any CUDA call
    lib.qdvm_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int]
    h = ctypes.c_void_p()
    assert lib.qdvm_plan_create(ctypes.byref(h), 4, 16, 3, 8.0, 0) == 1
    assert lib.qdvm_plan_create(ctypes.byref(h), 2, 2, 3, 8.0, 0) == 1
    assert lib.qdvm_plan_create(ctypes.byref(h), 2, 16, 0, 8.0, 0) == 1
    assert lib.qdvm_plan_create(ctypes.byref(h), 2, 16, 3, -1.0, 0) == 1
    lib.qdvm_plan_destroy.argtypes = [ctypes.c_void_p]
    assert lib.qdvm_plan_destroy(None) == 0
