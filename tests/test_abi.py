"""The C ABI library builds for sm_103a, loads, and exports every function
declared in include/aqr.h (no compute calls: this runs without a GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "aqr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aqr_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_query_path():
    names = _declared()
    for must in ("aqr_quantize", "aqr_load_graph", "aqr_search", "aqr_submit", "aqr_poll"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2602_21600_gb300 import aqr
    path = aqr.library_path()
    aqr.lib()  # builds if needed
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(aqr_[a-z0-9_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert set(_declared()) == set(aqr.SIGNATURES)


def test_checked_library_exports_every_declared_symbol():
    # the bounds-checked build (-DAQR_CHECKED) has the same C ABI
    from paper_2602_21600_gb300 import aqr
    from paper_2602_21600_gb300 import build as b
    path = b.build_library(checked=True)
    assert path.endswith("libaqr_checked.so") and os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(aqr_[a-z0-9_]+)\b", out))
    assert not [n for n in _declared() if n not in exported]
    L = aqr.lib(checked=True)
    assert L.aqr_status_string(0) == b"ok"


def test_status_strings_without_gpu():
    from paper_2602_21600_gb300 import aqr
    L = aqr.lib()
    assert L.aqr_status_string(0) == b"ok"
    assert L.aqr_status_string(6) == b"bad index file"
    # no device here: creating a context fails with a status, not a crash
    h = ctypes.c_void_p()
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except ImportError:
        pass
    assert L.aqr_create(ctypes.byref(h), 0) != 0
