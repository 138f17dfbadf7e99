"""GB300-native symmetry-adapted spin-1/2 exact diagonalization hot path.

* ``paper_2308_16712_gb300.ed``     -- ctypes binding of libed.so (include/ed.h)
* ``paper_2308_16712_gb300.build``  -- nvcc build of libed.so for sm_103a

The binding is imported on demand so that ``build`` works before the library
exists.
"""
__all__ = ["ed", "build"]
