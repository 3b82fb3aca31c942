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


def _null_args(fn):
    out = []
    for a in fn.argtypes:
        if a in (ctypes.c_float, ctypes.c_double):
            out.append(0.0)
        elif a in (ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t):
            out.append(0)
        else:
            out.append(None)
    return out


def test_every_entry_point_rejects_null_handles_without_a_device():
    """Status codes, not crashes, for null handles and pointers: every call checks
    its handle before it touches the device (FS4D_ERR_INVALID_ARG = 1)."""
    from paper_2310_08528_gb300 import build, fs4d
    build.build()
    lib = fs4d.library()
    fs4d._server_sigs(lib)
    checked = 0
    for name in declared_symbols():
        fn = getattr(lib, name)
        if name in ("fs4d_last_error", "fs4d_sort_pairs_noalloc") or fn.argtypes is None:
            continue
        rc = fn(*_null_args(fn))
        # freeing a null frame or trainer is a no-op, like free(NULL)
        assert rc == (0 if name in ("fs4d_frame_free", "fs4d_train_destroy") else 1), name
        checked += 1
    assert checked == len(declared_symbols()) - 2
    assert lib.fs4d_last_error(None) == b"null context"


def test_noalloc_sort_checks_sizes_before_any_device_call():
    """The allocation-free sort rejects bad sizes and returns early for n = 0
    without touching a device (FS4D_OK = 0, INVALID_ARG = 1, CAPACITY = 3)."""
    from paper_2310_08528_gb300 import build, fs4d
    build.build()
    lib = fs4d.library()
    f = lib.fs4d_sort_pairs_noalloc
    assert f(None, 0, 32, None, None) == 0
    assert f(None, -1, 32, None, None) == 1
    assert f(None, 10, 0, None, None) == 1
    assert f(None, 10, 65, None, None) == 1
    assert f(None, 10, 32, None, None) == 1
    big = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert f(None, (1 << 20) + 1, 32, big, big) == 3


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes across the boundary has the size, field
    names and field offsets that a C compiler gives the declaration in
    include/fs4d.h (compiled here with gcc; no GPU)."""
    import subprocess
    from paper_2310_08528_gb300 import fs4d
    pairs = [("fs4d_scene_desc", fs4d.SceneDesc), ("fs4d_camera", fs4d.Camera), ("fs4d_projected", fs4d.Projected),
             ("fs4d_grads", fs4d.Grads), ("fs4d_server_config", fs4d.ServerConfig), ("fs4d_request", fs4d.Request),
             ("fs4d_completion", fs4d.Completion), ("fs4d_server_stats", fs4d.ServerStats)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fs4d.h"', "int main(void) {"]
    for cname, py in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    for cname, py in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_binding_argument_types_match_the_prototypes():
    """Each ctypes signature in the binding has the prototype's argument count,
    with a pointer where the header has one and the same integer or float width
    elsewhere (enums and fs4d_scene_id are 32-bit)."""
    from paper_2310_08528_gb300 import build, fs4d
    build.build()
    lib = fs4d.library()
    fs4d._server_sigs(lib)
    src = open(os.path.join(ROOT, "include", "fs4d.h")).read()
    scalar = {"int32_t": ctypes.c_int32, "int": ctypes.c_int32, "fs4d_scene_id": ctypes.c_int32,
              "fs4d_precision": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
              "uint32_t": ctypes.c_uint32,
              "float": ctypes.c_float, "size_t": ctypes.c_size_t}
    protos = re.findall(r"FS4D_API\s+[\w\s\*]+?\b(fs4d_\w+)\s*\(([^)]*)\)\s*;", src)
    assert len(protos) == len(declared_symbols())
    for name, args in protos:
        fn = getattr(lib, name)
        decl = [a.strip() for a in " ".join(args.split()).split(",") if a.strip() and a.strip() != "void"]
        assert fn.argtypes is not None and len(fn.argtypes) == len(decl), name
        for a, t in zip(decl, fn.argtypes):
            if "*" in a:
                assert t is ctypes.c_void_p or t is ctypes.c_char_p or hasattr(t, "_type_") and \
                    issubclass(t, ctypes._Pointer), (name, a, t)
            else:
                base = a.replace("const ", "").split()[0]
                assert ctypes.sizeof(t) == ctypes.sizeof(scalar[base]), (name, a, t)
                assert (t in (ctypes.c_float, ctypes.c_double)) == (base == "float"), (name, a, t)


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, precisions, binning modes and the allocation-free sort's limit
    as the binding names them are the header's values."""
    import subprocess
    from paper_2310_08528_gb300 import fs4d
    consts = {name: code for code, name in fs4d.STATUS.items()}
    consts.update({"FS4D_FP32": fs4d.FP32, "FS4D_BF16": fs4d.BF16, "FS4D_BINNING_AUTO": fs4d.BINNING_AUTO,
                   "FS4D_BINNING_SORT": fs4d.BINNING_SORT, "FS4D_BINNING_BITMAP": fs4d.BINNING_BITMAP})
    src = tmp_path / "consts.c"
    body = "\n".join(f'  printf("{k} %lld\\n", (long long){k});' for k in consts)
    src.write_text(f'#include <stdio.h>\n#include "fs4d.h"\nint main(void) {{\n{body}\n'
                   f'  printf("FS4D_NOALLOC_MAX_PAIRS %lld\\n", (long long)FS4D_NOALLOC_MAX_PAIRS);\n  return 0;\n}}\n')
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict((a, int(b)) for a, b in (ln.split() for ln in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()))
    for k, v in consts.items():
        assert got[k] == v, k
    assert set(fs4d.STATUS) == set(range(10))  # every fs4d_status value has a name in the binding
    assert got["FS4D_NOALLOC_MAX_PAIRS"] == 1 << 20


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: with the shared library missing, loading it raises."""
    import pytest
    from paper_2310_08528_gb300 import fs4d
    with pytest.raises(RuntimeError, match="missing"):
        fs4d.library(str(tmp_path / "libfs4d.so"))
