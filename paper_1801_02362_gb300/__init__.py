"""GB300-native batched path-CV / MSD library (C ABI in include/pcv.h).

Mean-square-distance evaluation behind property-map / path collective variables with
the floating close-structure approximation of Pazurikova et al. (arXiv:1801.02362):
hand-written sm_103a CUDA kernels in ``csrc/`` built into ``_build/libpcv.so``, a ctypes
binding in ``pcv.py`` and seeded synthetic inputs in ``synth.py``.
"""
__all__ = ["pcv", "synth", "build_lib"]
