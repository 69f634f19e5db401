"""Write the oracle fixtures of tests/golden/ (calls only oracle/ and the
seeded input generators; never the CUDA path).

    python tests/golden/make_golden.py

config1_oracle.json: the FP64 oracle's result on the 32^3 sphere + box
union (k = 10, the paper's 2D search parameters): element counts, digests
of the integer results (1D results T, triangles, quad cases) and the first
vertices, so that any later change of the oracle's arithmetic shows up
against a stored record.
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(np.asarray(a, np.int64)).tobytes()).hexdigest()


def config1_record():
    from oracle import odc as oracle
    from paper_2409_13418_gb300 import inputs as I
    r = oracle.extract(I.config1_csg(), I.cube_grid(32), steps_1d=10)
    return {
        "what": "FP64 oracle, 32^3 cells on [-1,1]^3, union of sphere r 0.55 at (0.1,0,0) and AABB half 0.35 at "
                "(-0.3,0.2,0), iso 0.5, k = 10, 2D search (4 + 11, 0.8) and (3 + 12, sqrt(2)/2)",
        "counts": {"edges": int(len(r.edges)), "face_segments": int(len(r.faces)), "cells": int(len(r.cells)),
                   "verts3": int(len(r.verts_local)), "case3": int(np.sum(r.quad_case == 3)),
                   "flips": int(len(r.flips)), "vertices": int(len(r.vertices)), "triangles": int(len(r.triangles))},
        "sha256": {"edges": digest(r.edges), "T": digest(r.T), "triangles": digest(r.triangles),
                   "quad_case": digest(r.quad_case), "configs": digest(r.configs)},
        "first_vertices": [[round(float(x), 9) for x in v] for v in r.vertices[:16]],
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "config1_oracle.json"), "w") as f:
        json.dump(config1_record(), f, indent=1)
        f.write("\n")
    print("wrote", os.path.join(HERE, "config1_oracle.json"))
