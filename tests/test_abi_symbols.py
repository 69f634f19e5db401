"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/odc.h (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "odc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(odc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("odc_ctx_create", "odc_ctx_destroy", "odc_extract", "odc_mesh_copy", "odc_mesh_release",
                 "odc_source_upload", "odc_debug_copy", "odc_eval_points", "odc_status_str", "odc_last_error",
                 "odc_compact_edges_noalloc", "odc_launch_count"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2409_13418_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # exported names match the header exactly
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r" T (odc_[a-z0-9_]+)$", out, flags=re.M)))
    assert exported == declared_functions()


def test_status_strings_without_gpu():
    from paper_2409_13418_gb300 import odc
    lib = odc.load()
    assert lib.odc_status_str(0) == b"ok"
    assert lib.odc_status_str(2) == b"out of memory"


def test_binding_refuses_missing_library(tmp_path):
    from paper_2409_13418_gb300 import odc
    import pytest
    with pytest.raises(RuntimeError):
        odc.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(odc.load, "__wrapped__") else \
            _load_fresh(str(tmp_path / "nope.so"))


def _load_fresh(path):
    from paper_2409_13418_gb300 import odc
    saved = odc._lib
    odc._lib = None
    try:
        return odc.load(path)
    finally:
        odc._lib = saved
