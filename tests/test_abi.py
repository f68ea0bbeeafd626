"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/dgs.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:dgs_status|void|const char \*)\s*\*?\s*(dgs_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dgs_create", "dgs_scene_upload", "dgs_camera_set", "dgs_render", "dgs_render_backward",
                 "dgs_submit", "dgs_poll"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2508_03180_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2508_03180_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.exported_symbols())


def test_struct_sizes_match_the_header():
    """ctypes mirrors have the C layout (checked against a tiny C program)."""
    import subprocess
    import tempfile
    from paper_2508_03180_gb300 import _lib as L
    prog = r'''
#include <stdio.h>
#include "dgs.h"
#include <stddef.h>
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dgs_config), sizeof(dgs_scene_desc),
         sizeof(dgs_camera), sizeof(dgs_stats), sizeof(dgs_grads), sizeof(dgs_request), sizeof(dgs_result),
         offsetof(dgs_request, out_rgb), sizeof(dgs_serve_stats), sizeof(dgs_compare_config),
         offsetof(dgs_compare_config, w_bg), sizeof(dgs_neural_desc), offsetof(dgs_scene_desc, neural));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        got = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(L.dgs_config), ctypes.sizeof(L.dgs_scene_desc), ctypes.sizeof(L.dgs_camera),
            ctypes.sizeof(L.dgs_stats), ctypes.sizeof(L.dgs_grads), ctypes.sizeof(L.dgs_request),
            ctypes.sizeof(L.dgs_result), L.dgs_request.out_rgb.offset, ctypes.sizeof(L.dgs_serve_stats),
            ctypes.sizeof(L.dgs_compare_config), L.dgs_compare_config.w_bg.offset, ctypes.sizeof(L.dgs_neural_desc),
            L.dgs_scene_desc.neural.offset]
    assert got == want
