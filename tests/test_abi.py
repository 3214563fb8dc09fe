"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/dd.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:dd_status|int32_t|const char \*)\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dd_setup", "dd_apply", "gmres_solve", "dd_destroy", "dd_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1104_3349_gb300 import dd
    path = dd.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), f"libdd.so does not export {name}"
    assert sorted(dd.EXPORTS) == declared_functions()


def test_setup_rejects_bad_arguments_without_gpu_work():
    """Argument validation runs on the host before any device call."""
    from paper_1104_3349_gb300 import dd
    lib = dd.load(dd.build())
    h = ctypes.c_void_p()
    rc = lib.dd_setup(None, None, 1, None, None, ctypes.byref(h))
    assert rc == 1 and not h.value
    assert b"required" in lib.dd_last_error(None)
