"""The C-ABI library builds, loads and exports every entry point of jn.h
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1904_11201_gb300 import build as B
from paper_1904_11201_gb300 import jn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build()


def header_functions():
    text = open(os.path.join(ROOT, "include", "jn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"typedef\s+\w+\s*\(\s*\*\s*\w+\s*\)\s*\([^)]*\)\s*;", "", text)  # function-pointer types
    names = re.findall(r"\b(jn_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_binding_names():
    assert header_functions() == jn.exported_symbols()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (jn_[a-z_0-9]+)\b", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_without_gpu(lib_path):
    lib = jn.load(lib_path)
    assert lib.jn_version().startswith(b"jn ")
    assert lib.jn_status_str(jn.JN_ERR_CAPACITY) == b"output buffer too small"
    # NULL context arguments are rejected without touching a device
    assert lib.jn_set_profiling(None, 1) == jn.JN_ERR_INVALID
    assert lib.jn_count(None, 0, None, None, None, None) == jn.JN_ERR_INVALID
    assert lib.jn_sort_merge(None, None, None, None, 0, None) == jn.JN_ERR_INVALID
    assert lib.jn_selftest_wait(None, 1, 0, None) == jn.JN_ERR_INVALID
    assert lib.jn_autotune(None, jn.JN_ALGO_SORT, None, None, None, None) == jn.JN_ERR_INVALID
    assert lib.jn_server_wait_any(None, None, None, 0) == jn.JN_ERR_INVALID
    assert lib.jn_star(None, None, None, None, None, 0, None) == jn.JN_ERR_INVALID
    assert lib.jn_star_count(None, None, None, None, None) == jn.JN_ERR_INVALID
    # a server configuration is checked before any device is touched: the
    # small-request lane must leave at least one slot for large requests
    srv = ctypes.c_void_p()
    for slots, small, hold in ((4, 4, 0), (4, -1, 0), (1, 1, 0), (2, 0, -1)):
        cfg = jn.ServerConfig(slots, 1 << 18, 8, 0, 1 << 30, small, hold, 0, 0)
        assert lib.jn_server_create(ctypes.byref(srv), 0, ctypes.byref(cfg)) == jn.JN_ERR_INVALID
    h = ctypes.c_void_p()
    st = lib.jn_create(ctypes.byref(h), 0, None)
    # no GPU in this container: creation must fail cleanly, not crash
    import torch
    if not torch.cuda.is_available():
        assert st != jn.JN_OK and not h.value


def test_build_targets_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly():
    # the product path has no fallback: without libjn.so the binding raises
    code = ("from paper_1904_11201_gb300 import jn\n"
            "try:\n    jn.load('/nonexistent/libjn.so')\nexcept RuntimeError as e:\n"
            "    print('raised', 'not found' in str(e))\n")
    out = subprocess.run(["python", "-c", code], capture_output=True, text=True, cwd=ROOT).stdout
    assert out.strip() == "raised True"
