"""Plain FP64 CPU oracle of occupancy-based dual contouring (ODC).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path; the two meet only in the seeded input generators
(``paper_2409_13418_gb300.inputs``), which hold none of the method's
arithmetic.

Modules:
  occupancy  -- phi(p) for CSG and MLP sources, with decision margins (Sec. 3, A.2.2)
  topology   -- cube tables, face pairing, cycles and the manifold fix (A.1.1)
  odc        -- the ODC pipeline: crossings (Sec. 3), 1D search (Sec. 5.1),
                2D search (Sec. 5.2, A.1.3-A.1.4), normals (Sec. 5.3),
                QEF (Eq. 2), quads with IC splitting (Sec. 5.4, A.1.5)
  meshcheck  -- manifold / watertight / Euler / volume checks of a mesh
  quality    -- Sec. 6.1 metrics: |phi - 0.5| on area-uniform mesh samples
                (counter-based SplitMix64) and self-intersecting triangle pairs
"""
