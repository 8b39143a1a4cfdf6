"""GB300-native time-reversible FDTD gradients with a compressed boundary tape.

Modules:
  inputs  -- seeded synthetic workloads (no method arithmetic)
  _capi   -- ctypes binding of include/fdtd.h
  fdtd    -- Simulation handle and the FDTDGrad autograd Function
  build   -- nvcc build of the sm_103a library
"""
__all__ = ["inputs", "build"]


def __getattr__(name):
    if name in ("fdtd", "_capi"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
