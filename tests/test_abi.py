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
    lib = dvm.lib()
    for n in declared_functions():
        assert getattr(lib, n).argtypes is not None or getattr(lib, n).restype is not None, n


def test_status_strings_without_gpu():
    assert dvm.status_string(dvm.DVM_OK) == "DVM_OK"
    assert dvm.status_string(dvm.DVM_ERR_ADMISSION) == "DVM_ERR_ADMISSION"


def test_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
