"""The C-ABI library builds for sm_103a, loads, and exports every function
``include/polylla.h`` declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re
import subprocess

import numpy as np

import pytest

from paper_2403_14723_gb300 import build, polylla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polylla.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(polylla_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("polylla_create", "polylla_generate", "polylla_get_polygons", "polylla_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(polylla_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_every_symbol():
    assert set(declared_functions()) == set(polylla._SIGNATURES)


def test_status_strings_without_gpu(lib_path):
    lib = polylla.load_library()
    assert lib.polylla_status_string(0) == b"ok"
    assert lib.polylla_status_string(-2) == b"invalid mesh layout"
    assert lib.polylla_stage_count() == 8
    names = [lib.polylla_stage_name(i).decode() for i in range(8)]
    assert lib.polylla_stage_name(8) == b""
    assert names == ["longest_edge", "label_relink", "chords", "chord_links", "poly_count", "tile_scan",
                     "poly_list", "batch_meta"]


def test_null_arguments_rejected_without_gpu(lib_path):
    lib = polylla.load_library()
    ctx = ctypes.c_void_p()
    assert lib.polylla_create(None, None, None, None) == -1
    assert lib.polylla_create(ctypes.byref(ctx), None, None, None) == -1
    m = polylla.polylla_mesh(3, 1, 2, None, None, None, None, None)   # H < 3T + 3
    assert lib.polylla_create(ctypes.byref(ctx), ctypes.byref(m), None, None) == -1
    assert lib.polylla_generate(None, None) == -1
    assert lib.polylla_get_polygons(None, None, None) == -1
    m = polylla.polylla_mesh(3, 0, 3, 16, 16, 16, 16, 16)                # no triangles
    assert lib.polylla_create(ctypes.byref(ctx), ctypes.byref(m), None, None) == -1
    T = 715_827_883                                                      # 3T no longer fits int32
    m = polylla.polylla_mesh(T + 2, T, 2 ** 31 - 1, 16, 16, 16, 16, 16)
    assert lib.polylla_create(ctypes.byref(ctx), ctypes.byref(m), None, None) == -1
    assert lib.polylla_create_host(ctypes.byref(ctx), 3, 0, 3, None) == -1
    assert lib.polylla_batch_create(None, None, None, None) == -1
    assert lib.polylla_batch_create(ctypes.byref(ctx), None, None, None) == -1
    one = np.array([0, 3], dtype=np.int32)
    zero_t = np.array([0, 0], dtype=np.int32)                          # a mesh without triangles
    b = polylla.polylla_batch(1, one.ctypes.data, zero_t.ctypes.data, one.ctypes.data, 16, 16, 16, 16, 16)
    assert lib.polylla_batch_create(ctypes.byref(ctx), ctypes.byref(b), None, None) == -1
    assert lib.polylla_capture_graph(None, None) == -1
    assert lib.polylla_autotune(None, 1, None, None) == -1
    assert lib.polylla_set_tuning(None, None) == -1
    assert lib.polylla_batch_polygon_offsets(None, None) == -1
    assert lib.polylla_tuning_cache_clear() == 0
    srv = ctypes.c_void_p()
    assert lib.polylla_server_create(None, None) == -1
    assert lib.polylla_server_create(ctypes.byref(srv), None) == -1
    bad = polylla.polylla_server_options(0, 3, 0, 0, 0)                  # no memory budget
    assert lib.polylla_server_create(ctypes.byref(srv), ctypes.byref(bad)) == -1
    bad = polylla.polylla_server_options(1 << 30, 99, 0, 0, 0)           # too many slots
    assert lib.polylla_server_create(ctypes.byref(srv), ctypes.byref(bad)) == -1
    assert lib.polylla_server_submit(None, None, None) == -1
    assert lib.polylla_server_get_stats(None, None) == -1
    assert lib.polylla_server_get_batch_log(None, None, 0, None, None) == -1
    assert lib.polylla_server_replay(None, 0, None, None, None, None) == -1


def test_built_for_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the built library every call raises."""
    with pytest.raises(RuntimeError, match="not built"):
        polylla.load_library(str(tmp_path / "libpolylla_missing.so"))


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets (a C program built from include/polylla.h prints them)."""
    import shutil

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(polylla, n) for n in dir(polylla)
               if n.startswith("polylla_") and isinstance(getattr(polylla, n), type)
               and issubclass(getattr(polylla, n), ctypes.Structure)]
    assert len(structs) >= 13
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "polylla.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'    printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(build.ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                                text=True).stdout.splitlines())
    for st in structs:
        name = st.__name__
        assert int(got[name]) == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(st, f).offset, f"{name}.{f}"
