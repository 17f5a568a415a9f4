"""CPU-side checks of the C ABI: the library builds, loads and exports every declared entry point.
No compute call is made (no GPU here)."""
import ctypes
import os
import re

from paper_2501_00923_gb300 import build, dvm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dvm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dvm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_names():
    """Every declared entry point has an explicit signature in the binding (ctypes' defaults, no
    argtypes and an int result, would let a wrong call through)."""
    from paper_2501_00923_gb300 import serve
    lib = serve._bind()             # the served-batch calls are bound by serve.py, the rest by dvm.py
    unbound = [n for n in declared_functions() if getattr(lib, n).argtypes is None]
    assert not unbound, unbound


def test_status_strings_without_gpu():
    assert dvm.status_string(dvm.DVM_OK) == "DVM_OK"
    assert dvm.status_string(dvm.DVM_ERR_ADMISSION) == "DVM_ERR_ADMISSION"


def test_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
