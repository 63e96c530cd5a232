"""GB300-native data-parallel volume rendering: per-brick emission-absorption
ray marching and sort-last "over" compositing (Sec. 2.2, 3 and 4 of
arXiv:2501.01628), as CUDA kernels for sm_103a behind a C-ABI library.

``synth`` generates seeded inputs; ``vr`` is the thin ctypes binding of
``libvr.so`` (it raises if the library has not been built)."""
from . import synth  # noqa: F401
