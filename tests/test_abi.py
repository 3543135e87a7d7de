"""The C-ABI library builds, loads and exports every declared entry point (no GPU).

Only host-side arithmetic and argument checks that return before any CUDA call
are exercised here; compute calls need a GPU and live in the gpu-marked tests.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1004_2772_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "reach.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return binding.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ht_create", "ht_find_or_put", "reach", "reach_ctx_run", "ht_scan"):
        assert n in names
    assert set(names) == set(binding.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_sizes_are_host_arithmetic(lib):
    nb = 1 << 20
    b = binding.ht_bytes(20, 16)
    assert b >= nb * 4 + nb * 64
    assert binding.ht_bytes(20, 5) >= nb * 4 + nb * 32  # rows padded to 16 bytes
    r = binding.reach_ctx_bytes(20, 16, 1024)
    assert r >= b + 2 * nb * 4 + 1024 * 8


def test_invalid_arguments_return_before_any_device_call(lib):
    out = ctypes.c_uint64()
    assert lib.ht_bytes(3, 16, ctypes.byref(out)) == binding.HT_ERR_INVALID
    assert lib.ht_bytes(20, 33, ctypes.byref(out)) == binding.HT_ERR_INVALID
    assert lib.ht_bytes(32, 1, ctypes.byref(out)) == binding.HT_ERR_INVALID
    assert lib.reach_ctx_bytes(20, 16, 0, ctypes.byref(out)) == binding.HT_ERR_INVALID
    h = ctypes.c_void_p()
    assert lib.ht_create(2, 16, None, ctypes.byref(h)) == binding.HT_ERR_INVALID
    assert lib.ht_find_or_put(None, None, 0, None, None, None) == binding.HT_ERR_INVALID
    assert lib.reach_ctx_run(None, 0, None) == binding.HT_ERR_INVALID
    ms = ctypes.c_float()
    assert lib.vss_probe_random_cfg(None, 1 << 30, 1 << 20, 0, 8, 8, 256, None,
                                    ctypes.byref(ms)) == binding.HT_ERR_INVALID
    assert lib.vss_probe_random(None, 1 << 30, 1 << 20, 8, None, ctypes.byref(ms)) == binding.HT_ERR_INVALID
    assert lib.ht_status_string(binding.HT_ERR_FULL).decode().startswith("table full")


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.load("/nonexistent/libvss.so")


def test_product_path_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1004_2772_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "oracle.cpp" not in text and "liboracle" not in text, f
    ora = open(os.path.join(ROOT, "oracle", "oracle.cpp")).read()
    assert "#include \"" not in ora  # the oracle includes no project header
