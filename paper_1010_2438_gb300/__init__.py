"""GB300-native batched Gillespie simulation of CWC rewrite systems.

Submodules:
  workloads  seeded synthetic models and batches (no simulation arithmetic)
  capi       ctypes binding of the C ABI (include/cwcgpu.h)
  api        torch device buffers, streams, autograd (MeanObservables)
  build      in-tree build of the sm_103a CUDA library

Importing the package does not load the CUDA library; ``capi.lib()`` does,
and raises if the library has not been built.
"""

__all__ = ["workloads", "capi", "api", "build"]
