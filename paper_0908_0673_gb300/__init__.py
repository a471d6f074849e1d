"""GB300-native FMM-accelerated collocation BEM (Carley, BEM3D).

The compute path lives in the CUDA library under ``csrc/`` behind the C ABI of
``include/bem.h``; ``paper_0908_0673_gb300.bem`` is the thin ctypes binding
with the same names.  ``inputs`` holds the seeded synthetic meshes and
boundary data shared by the tests, the benchmark and the oracle.
"""
