"""GB300-native batched lower-bound engine for certified k-sparse GLM branch and bound.

The compute path is the C-ABI library ``libkglm.so`` (CUDA, sm_103a) declared
in ``include/kglm.h``; ``paper_2605_22188_gb300.kglm`` is its thin ctypes
binding and ``paper_2605_22188_gb300.synth`` the seeded input generator.
Importing the package itself loads nothing.
"""

__all__ = ["kglm", "synth", "build"]
