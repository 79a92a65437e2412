"""CPU checks of the boundary: the C-ABI library builds for sm_103a, loads, and exports every
function include/ile.h declares.  No compute call is made (there is no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:ile_status|const\s+char\s*\*|int|void)\s*\**\s*(ile_\w+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2210_07912_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("ile_create", "ile_destroy", "ile_set_data", "ile_eval", "ile_integrate", "ile_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ile_\w+)$", out, re.M))
    assert set(declared_symbols()) <= exported


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.ile_status_string.restype = ctypes.c_char_p
    assert lib.ile_status_string(0) == b"ok"
    assert b"range" in lib.ile_status_string(3)
    lib.ile_destroy.argtypes = [ctypes.c_void_p]
    assert lib.ile_destroy(None) == 0


def test_create_rejects_bad_arguments_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.ile_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    h = ctypes.c_void_p()
    assert lib.ile_create(ctypes.byref(h), 0, None, 7) == 1  # bad precision -> ILE_E_ARG
    assert lib.ile_create(None, 0, None, 0) == 1
    assert not h

