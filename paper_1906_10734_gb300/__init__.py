"""GB300 (sm_103a) solver for the Hierarchical Particle-Mesh FMM (Gnedin 2019).

The compute path is the CUDA library ``_build/libhpm.so`` behind the C ABI in
``include/hpm.h``; the submodule ``hpm`` is its ctypes binding and ``inputs``
holds the seeded synthetic particle sets. Submodules are imported on demand,
so the input generators work without a built library.
"""
