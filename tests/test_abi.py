"""The C-ABI library builds, loads on a machine without a GPU and exports every function
that include/hz.h declares (no compute calls here)."""
import os
import re

import paper_1811_12378_gb300 as hzpkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\**\s*\**\s*(hz_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_binding_exports():
    decl = declared_functions()
    assert len(decl) >= 12
    assert sorted(hzpkg.EXPORTS) == decl


def test_library_exports_every_declared_symbol():
    lib = hzpkg.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert lib.hz_status_string(0).decode() == "ok"
    assert lib.hz_status_string(4).decode() == "not converged"
    assert isinstance(lib.hz_launch_count(), int)


def test_invalid_arguments_are_rejected_without_a_gpu():
    """Argument checks happen before any CUDA call."""
    import ctypes as C
    lib = hzpkg.load()
    h = C.c_void_p()
    assert lib.hz_problem_create(None, None, None, None, C.byref(h)) == 1
    assert lib.hz_problem_destroy(None) == 0
    assert lib.hz_plan(None, None, None, None, None, None, None, None, None, None, None) == 1
    assert b"invalid" in lib.hz_last_error()
