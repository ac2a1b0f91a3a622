"""Flexible shifted-Krylov solver for GB300 (sm_103a).

The compute path is libfks.so (CUDA, built by paper_1212_3660_gb300.build)
behind the C ABI of include/fks.h; `fks` is its ctypes binding, `solver` a
convenience layer, `synth` the seeded synthetic-aquifer generator.
"""
__all__ = ["fks", "solver", "synth", "build"]
