"""The C-ABI library builds, loads and exports every entry point its header declares."""
import ctypes
import os
import re
import subprocess

import paper_2605_07391_gb300 as mb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(merbit_\w+)\s*\(", src))
    return names


def test_library_exports_declared_symbols():
    lib = mb.load()
    declared = _declared()
    assert declared == set(mb.EXPORTS), declared ^ set(mb.EXPORTS)
    for name in declared:
        assert getattr(lib, name) is not None
    assert mb.version().startswith("merbit-gb300")


def test_exported_symbols_have_c_linkage():
    out = subprocess.run(["nm", "-D", "--defined-only", mb.library_path()],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(merbit_\w+)\b", out))
    assert _declared() <= exported


def test_errors_without_device_work():
    lib = mb.load()
    # argument checks reject before touching the device
    h = ctypes.c_void_p()
    st = lib.merbit_plan_ex(None, None, 10, 10, 0, 14, 8, None, ctypes.byref(h))
    assert st == 1 and b"row_ptr" in lib.merbit_last_error()
    st = lib.merbit_plan_ex(ctypes.c_void_p(16), None, -1, 10, 0, 14, 8, None, ctypes.byref(h))
    assert st == 1
    st = lib.merbit_plan_ex(ctypes.c_void_p(16), ctypes.c_void_p(16), 10, 10, 5, 43, 8, None,
                            ctypes.byref(h))
    assert st == 1 and b"sigma" in lib.merbit_last_error()
    st = lib.merbit_plan_ex(ctypes.c_void_p(16), ctypes.c_void_p(16), 2**30, 2**30, 2**30, 14, 8,
                            None, ctypes.byref(h))
    assert st == 2
    assert lib.merbit_spmv(None, 0, None, None, None) == 1
    assert lib.merbit_pagerank(None, 0, None, 0.85, 1e-10, None) == 1
    assert lib.merbit_plan_set_kernel(None, 2) == 1 and b"plan" in lib.merbit_last_error()
    lib.merbit_plan_destroy(None)
