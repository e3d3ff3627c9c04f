"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/ccov.h declares (no compute call here)."""
import ctypes
import os
import re

from paper_1808_02414_gb300 import build, ccov, surrogate

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header=None):
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h") or (header and h != header):
            continue
        with open(os.path.join(inc, h)) as f:
            names |= set(re.findall(r"CCOV_API[^;(]*?\b(ccov_\w+)\s*\(", f.read(), flags=re.S))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["ccov_create", "ccov_information", "ccov_schur", "ccov_nullspace",
                     "ccov_covariance", "ccov_destroy"]:
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(ccov.EXPORTED) == declared_symbols("ccov.h")
    assert sorted(surrogate.EXPORTED) == declared_symbols("ccov_surrogate.h")


def test_status_strings_without_gpu():
    L = ccov.load()
    assert L.ccov_status_string(0) == b"ok"
    assert L.ccov_status_string(2) == b"degenerate input"
