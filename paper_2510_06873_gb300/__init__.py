"""GB300 (sm_103a) metadynamics bias path behind a C ABI (include/metad.h).

Submodules:
  build   -- nvcc build of libmetad.so (in-tree)
  metad   -- ctypes binding with the C entry-point names
  autograd -- torch.autograd.Function whose backward is the adjoint kernel
  batch   -- many systems per launch
  serve   -- continuous-batching request loop for concurrent walkers
Importing the package loads nothing; the binding loads the library on first use.
"""
__all__ = ["build", "metad"]
