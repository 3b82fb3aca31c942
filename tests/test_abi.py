"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/fs4d.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fs4d.h")).read()
    return sorted(set(re.findall(r"FS4D_API\s+[\w\s\*]+?\b(fs4d_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("fs4d_load_scene", "fs4d_deform", "fs4d_render", "fs4d_render_backward"):
        assert n in names
    from paper_2310_08528_gb300 import fs4d
    assert sorted(fs4d.EXPORTS) == names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2310_08528_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_errors_without_gpu_are_reported_not_raised():
    """Creating a context with no usable device returns an error status."""
    from paper_2310_08528_gb300 import build, fs4d
    build.build()
    lib = fs4d.library()
    h = ctypes.c_void_p()
    rc = lib.fs4d_create(10_000, None, ctypes.byref(h))
    assert rc == 1 and not h.value
    assert lib.fs4d_destroy(None) == 1
