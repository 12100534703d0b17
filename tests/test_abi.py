"""The C-ABI library builds, loads and exports every entry point its header declares (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_24514_gb300 import build
    build.build()
    import paper_2605_24514_gb300 as pkg
    return pkg.lib()


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(isvd_\w+)\s*\(", src, re.M))
    return names


def test_header_declares_api():
    d = declared()
    for n in ["isvd_create", "isvd_append_row", "isvd_append_col", "isvd_update_entry", "isvd_refresh",
              "isvd_metrics", "isvd_destroy"]:
        assert n in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.isvd_status_string(0) == b"ok"
    assert lib.isvd_status_string(3) == b"index out of bounds"


def test_null_handle_is_rejected_without_gpu(lib):
    import ctypes as C
    assert lib.isvd_update_entry(None, 0, 0, 1.0) == 1      # EINVAL, no CUDA call made
    assert lib.isvd_sync(None) == 1
