"""GB300-native photon-conserving adaptive ray tracing (arXiv:1012.2865).

The computation lives in librt_gb300.so (CUDA kernels for sm_103a) behind the
C ABI of include/rt.h; ``native`` is its ctypes binding, ``synth`` draws the
seeded synthetic workloads, ``build`` compiles the library in-tree.
"""
