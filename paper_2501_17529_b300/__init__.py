"""B300-native batched DC loadflow over many grid topologies (arXiv 2501.17529).

* ``paper_2501_17529_b300.dcflow`` -- ctypes binding of libdcflow.so (the C ABI
  declared in include/dcflow.h); loads the library lazily and fails loudly if
  it has not been built.
* ``paper_2501_17529_b300.synth`` -- seeded synthetic grids, topologies,
  injections and injection candidates.
* ``paper_2501_17529_b300.csrc.build`` -- in-tree nvcc build for sm_103a.
"""
__all__ = ["dcflow", "synth"]
