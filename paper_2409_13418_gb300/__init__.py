"""GB300-native occupancy-based dual contouring (ODC).

``paper_2409_13418_gb300.odc`` binds the CUDA library (libodc.so);
``paper_2409_13418_gb300.inputs`` draws seeded synthetic instances;
``paper_2409_13418_gb300.build`` compiles the library with nvcc for sm_103a.
Importing the package itself loads nothing.
"""
