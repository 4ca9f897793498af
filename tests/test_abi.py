"""The C ABI on the host (no GPU): the library builds and loads, exports every entry point that
include/*.h declares, and rejects malformed meshes before touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vof():
    from paper_2604_14938_gb300 import build as b
    b.build()
    import paper_2604_14938_gb300 as p
    return p


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(vof_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(vof):
    L = vof.lib()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def _desc(vof, m):
    keep = [np.ascontiguousarray(a, dt) for a, dt in (
        (m.cell_face_off, np.int64), (m.cell_face, np.int32), (m.face_vert_off, np.int64), (m.face_vert, np.int32),
        (m.face_owner, np.int32), (m.face_neigh, np.int32), (m.vx, np.float64), (m.vy, np.float64),
        (m.vz, np.float64))]
    return keep, vof._Desc(len(keep[0]) - 1, len(keep[4]), len(keep[6]), *[a.ctypes.data for a in keep])


@pytest.mark.parametrize("corrupt", ["owner_range", "face_vert_range", "orientation", "nan_vertex", "short_face"])
def test_malformed_mesh_rejected_on_host(vof, corrupt):
    m = synth.hex_box(2)
    if corrupt == "owner_range":
        m.face_owner = m.face_owner.copy(); m.face_owner[3] = 99
    elif corrupt == "face_vert_range":
        m.face_vert = m.face_vert.copy(); m.face_vert[5] = -2
    elif corrupt == "orientation":
        m.cell_face = m.cell_face.copy(); m.cell_face[0] ^= np.int32(-2 ** 31)
    elif corrupt == "nan_vertex":
        m.vx = m.vx.copy(); m.vx[4] = np.nan
    elif corrupt == "short_face":
        m.face_vert_off = m.face_vert_off.copy(); m.face_vert_off[1] = 2
    keep, d = _desc(vof, m)
    h = ctypes.c_void_p()
    st = vof.lib().vof_mesh_create(ctypes.byref(d), None, ctypes.byref(h))
    assert st == 4, vof.lib().vof_last_error()
    assert not h.value
    assert vof.lib().vof_last_error()


def test_null_arguments(vof):
    L = vof.lib()
    assert L.vof_mesh_create(None, None, None) == 1
    assert L.vof_reconstruct(None, None, None, None) == 1
    assert L.vof_mesh_destroy(None) == 1
    o = vof.default_options()
    assert o.tol_alpha == 1e-12 and o.max_bisect == 100 and o.xf_mode == 0


def _c_layout(struct: str, fields: list[str], tmp_path) -> dict:
    """Offsets and size of a struct of include/vof.h, from a small C program compiled with gcc."""
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vof.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({struct}));']
    lines += [f'  printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("name", ["Options", "Counts", "Props", "_Desc"])
def test_struct_layouts_match_the_header(vof, name, tmp_path):
    """The binding's ctypes structures have the header's field offsets and size."""
    py = getattr(vof, name)
    struct = {"Options": "vof_options", "Counts": "vof_counts", "Props": "vof_props", "_Desc": "vof_mesh_desc"}[name]
    fields = [f for f, _ in py._fields_]
    c = _c_layout(struct, fields, tmp_path)
    assert c["size"] == ctypes.sizeof(py)
    for f in fields:
        assert c[f] == getattr(py, f).offset, f
