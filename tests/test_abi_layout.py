"""The ctypes structures of the binding have the layout of the C header's.

A C program compiled against include/odc.h prints the size of every public
structure and the offset of every field; the binding's ctypes mirrors must
agree on each (a field added to one side only would shift every later
field and corrupt calls silently).  Runs on the CPU with the host compiler.
"""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2409_13418_gb300 import odc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C type name -> binding structure; field names are the same on both sides
PAIRS = [
    ("odc_csg_prim", odc.Prim),
    ("odc_mlp", odc.Mlp),
    ("odc_voxels", odc.Voxels),
    ("odc_source", odc.Source),
    ("odc_grid", odc.Grid),
    ("odc_params", odc.Params),
    ("odc_stats", odc.Stats),
    ("odc_mesh", odc.MeshC),
    ("odc_slab", odc.SlabC),
    ("odc_slab_info", odc.SlabInfoC),
    ("odc_quality", odc.QualityC),
    ("odc_server_config", odc.ServerConfig),
    ("odc_result", odc.ResultC),
]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "odc.h"', "int main(void) {"]
    for cname, st in PAIRS:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in st._fields_:
            if f.startswith("pad"):
                continue
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    return got


def test_ctypes_structures_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for cname, st in PAIRS:
        assert c[(cname, "size")] == C.sizeof(st), cname
        for f, _ in st._fields_:
            if f.startswith("pad"):
                continue
            assert c[(cname, f)] == getattr(st, f).offset, (cname, f)
