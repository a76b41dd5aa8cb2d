"""GB300-native integral-histogram engine (Poostchi 2017, arXiv 1711.01656).

The compute path is the CUDA library ``libih.so`` (sources in ``csrc/``,
C ABI in ``include/ih.h``); ``ih`` is its ctypes binding and ``synth`` draws
seeded synthetic inputs.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "ih"]
