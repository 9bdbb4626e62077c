"""GB300 (sm_103a) library for one source iteration per time step of the
time-dependent, multi-group, mixed-frame relativistic SHDOM method
(Tominaga, Shibata & Blinnikov, arXiv:1507.05141).

The computation lives in a CUDA shared library with a C ABI
(``include/shdom_gb300.h``); :mod:`.native` is its ctypes binding and
:mod:`.inputs` draws seeded synthetic problems.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "native", "build"]
