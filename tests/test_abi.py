"""The C-ABI library loads and exports every symbol its header declares
(no compute calls; runs without a GPU)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"PG_API\s+[\w\s\*]*?\b(pg_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_api():
    names = _declared()
    for n in ("pg_fieldset_create", "pg_pset_create", "pg_kernel_create", "pg_execute",
              "pg_last_error"):
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1707_05163_gb300 import _native
    from paper_1707_05163_gb300 import build as build_mod
    path = build_mod.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pg_\w+)", out))
    assert set(_declared()) <= exported
    # the binding has a signature for every declared call
    assert set(_declared()) <= set(_native.exported_names())


def test_error_strings_without_gpu():
    from paper_1707_05163_gb300 import _native
    lib = _native.load()
    assert lib.pg_version().startswith(b"parcels-gb300")
    assert lib.pg_last_error() == b""
    # argument validation happens before any device call
    h = ctypes.c_void_p()
    r = lib.pg_kernel_create(7, 0, 0.0, 0.0, ctypes.byref(h))
    assert r == _native.PG_ERR_ARG
    assert b"scheme" in lib.pg_last_error()
    r = lib.pg_kernel_create(1, 0, -1.0, 0.0, ctypes.byref(h))
    assert r == _native.PG_ERR_ARG
