"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/gyps.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "gyps.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gyps_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1804_00995_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("gyps_mesh_create", "gyps_sl_assemble", "gyps_sl_apply", "gyps_near_correct",
                     "gyps_gmres_solve", "gyps_rhs_planewave", "gyps_mesh_destroy", "gyps_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib_path):
    import paper_1804_00995_gb300 as g
    assert set(declared_symbols()) == set(g._SIGS)
    lib = g.load(lib_path)
    assert lib.gyps_version().decode().startswith("gyps")


def test_invalid_arguments_are_rejected_without_a_gpu(lib_path):
    import numpy as np
    import paper_1804_00995_gb300 as g
    lib = g.load(lib_path)
    h = ctypes.c_void_p()
    vtx = np.zeros((3, 3))
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    # quadrature order 2 does not exist: rejected before any device work
    code = lib.gyps_mesh_create(vtx.ctypes.data, 3, tri.ctypes.data, 1, 2, 0, None, ctypes.byref(h))
    assert code == 1
    buf = ctypes.create_string_buffer(256)
    assert lib.gyps_last_error(buf, 256) == 1
    assert b"quad_points" in buf.value
    assert lib.gyps_sl_apply(None, 1.0, 1, None, 1, None, 1, 1, 0, -1, -1, None) == 1


STRUCTS = {"_MeshInfo": "gyps_mesh_info_t", "_Profile": "gyps_profile_t", "_BatchItem": "gyps_batch_item",
           "_BatchInfo": "gyps_batch_info_t", "_GmresOpts": "gyps_gmres_opts", "_GmresReport": "gyps_gmres_report",
           "_HmatInfo": "gyps_hmat_info_t"}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes mirror has the header struct's size and field offsets (gcc on the header)."""
    import shutil
    import subprocess
    import paper_1804_00995_gb300 as g
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "gyps.h"', "int main(void) {"]
    expect = []
    for py, c in STRUCTS.items():
        cls = getattr(g, py)
        lines.append(f'printf("%zu\\n", sizeof({c}));')
        expect.append(ctypes.sizeof(cls))
        for name, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({c}, {name}));')
            expect.append(getattr(cls, name).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
