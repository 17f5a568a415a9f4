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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the public structs have the C sizes and field offsets: a C program
    compiled against include/dvm.h prints them (gcc; no GPU)."""
    import shutil
    import subprocess
    from paper_2501_00923_gb300 import serve
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    pairs = [("dvm_options", dvm.Options), ("dvm_flow", dvm.Flow), ("dvm_solve_opts", dvm.SolveOpts),
             ("dvm_primal_result", dvm.PrimalResult), ("dvm_adjoint_result", dvm.AdjointResult),
             ("dvm_batch_options", serve.BatchOptions), ("dvm_request", serve.Request),
             ("dvm_request_result", serve.RequestResult), ("dvm_batch_stats", serve.BatchStats)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dvm.h"', 'int main(void) {']
    for cname, py in pairs:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
