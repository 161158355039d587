"""GB300-native ring-polymer PIMD (the "fix pimd/langevin" method).

Submodules:
  binding -- ctypes binding of the C ABI in include/pimd.h (libpimd.so)
  build   -- nvcc build of libpimd.so for sm_103a
  inputs  -- seeded synthetic workloads (no method arithmetic)
"""
from . import inputs  # noqa: F401

__all__ = ["binding", "build", "inputs"]
