"""GB300-native matrix-free P1 geometric multigrid on hierarchical hybrid grids.

* ``paper_1805_10167_gb300.hhg``    -- ctypes binding of libhhg.so (the CUDA path)
* ``paper_1805_10167_gb300.inputs`` -- seeded synthetic meshes, right-hand sides
  and coefficient fields
* ``paper_1805_10167_gb300.build``  -- nvcc build of libhhg.so for sm_103a

The binding is imported on demand so that the input generators stay usable on
machines where the library has not been built.
"""
