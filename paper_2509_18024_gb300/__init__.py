"""GB300-native core-elements ALS (Xue, Li, Zhang, Meng, arXiv 2509.18024).

Submodules:
  synth      seeded synthetic rating matrices and initial factors (numpy only)
  build      in-tree nvcc build of libcore_als.so (sm_103a)
  binding    ctypes declarations of the C ABI in include/core_als.h
  core_als   CoreALS / DeviceCSR: the Python front end (torch for memory)

Importing the package does not load CUDA; ``core_als`` does.
"""

__all__ = ["synth", "build", "binding", "core_als"]


def __getattr__(name):
    if name in ("CoreALS", "DeviceCSR"):
        from . import core_als
        return getattr(core_als, name)
    raise AttributeError(name)
