"""Stored fixtures (tests/golden/): the paper's printed search parameters,
and the oracle's record of the 32^3 sphere + box run.

* paper_parameters.json holds values the paper prints (cited per entry);
  the oracle's defaults, the binding's defaults and the C header's stated
  defaults must be those values, and the per-face evaluation count the
  paper gives must follow from them.
* config1_oracle.json is written by tests/golden/make_golden.py, which
  calls only the oracle: the oracle must still reproduce it exactly (a
  change to the oracle's arithmetic shows up here first), and on a GPU the
  CUDA path must give the same integers and vertices.
"""
import hashlib
import inspect
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_paper_parameters_are_the_defaults():
    from oracle import odc as oracle
    from paper_2409_13418_gb300 import odc
    P = {k: v["value"] for k, v in _load("paper_parameters.json").items() if isinstance(v, dict)}
    d = inspect.signature(oracle.extract).parameters
    assert d["iso"].default == P["iso"]
    assert (d["lin1"].default, d["bin1"].default, d["range1"].default) == \
        (P["step1_line_samples"], P["step1_binary_steps"], P["step1_range_cells"])
    assert (d["lin2"].default, d["bin2"].default) == (P["step2_line_samples"], P["step2_binary_steps"])
    assert abs(d["range2"].default - P["step2_range_cells"]) < 1e-7
    assert d["steps_1d"].default == P["bisection_steps_128"]
    b = inspect.signature(odc.make_params).parameters
    assert (b["iso"].default, b["lin1"].default, b["bin1"].default, b["lin2"].default, b["bin2"].default) == \
        (P["iso"], P["step1_line_samples"], P["step1_binary_steps"], P["step2_line_samples"], P["step2_binary_steps"])
    assert abs(b["range1"].default - P["step1_range_cells"]) < 1e-7
    assert abs(b["range2"].default - P["step2_range_cells"]) < 1e-7
    # the paper's per-face count: three line-binary searches of (samples + iterations)
    assert (P["step1_line_samples"] + P["step1_binary_steps"]) * 3 == P["evaluations_per_face"]
    assert P["step2_line_samples"] + P["step2_binary_steps"] == P["step1_line_samples"] + P["step1_binary_steps"]
    assert abs(P["step2_range_cells"] - math.sqrt(2) / 2) < 1e-15
    hdr = open(os.path.join(os.path.dirname(HERE), "..", "include", "odc.h")).read()
    assert "4 samples + 11 bisections over\n * 0.8 cell" in hdr and "3 samples + 12 bisections over sqrt(2)/2 cell" in hdr


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(np.asarray(a, np.int64)).tobytes()).hexdigest()


def test_oracle_reproduces_its_stored_record():
    import sys
    sys.path.insert(0, HERE)
    from make_golden import config1_record
    assert config1_record() == _load("config1_oracle.json")


@pytest.mark.gpu
def test_cuda_path_matches_the_stored_oracle_record():
    from paper_2409_13418_gb300 import build, inputs as I, odc
    build.build()
    g = _load("config1_oracle.json")
    with odc.Context(0) as ctx:
        m = ctx.extract(I.config1_csg(), I.cube_grid(32), steps_1d=10)
        v, t = m.to_host()
        assert _digest(ctx.debug("edges")) == g["sha256"]["edges"]
        assert _digest(ctx.debug("T")) == g["sha256"]["T"]
        assert _digest(ctx.debug("configs")) == g["sha256"]["configs"]
        assert _digest(t) == g["sha256"]["triangles"]
        assert (m.n_verts, m.n_tris) == (g["counts"]["vertices"], g["counts"]["triangles"])
        ref = np.asarray(g["first_vertices"])
        assert np.abs(v[:len(ref)] - ref).max() / (2.0 / 32) < 1e-4
