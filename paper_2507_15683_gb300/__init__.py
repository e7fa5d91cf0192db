"""GB300-native tile-based Gaussian-splatting rasterizer with se(3) pose gradient.

The compute path lives in the CUDA library ``libgsr.so`` built from ``csrc/``
(see ``build.py``); ``gsr`` is its thin ctypes binding. Importing this package
does not load the library; ``paper_2507_15683_gb300.gsr`` does, and raises if
it is missing.
"""
__all__ = ["gsr", "synth", "build"]
