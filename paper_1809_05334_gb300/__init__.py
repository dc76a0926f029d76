"""GB300-native preconditioned periodic volume-integral-equation solver.

The compute path is the CUDA library libvie.so (C ABI in include/vie.h); this
package holds its sources (csrc/), the in-tree build (build.py) and a thin
ctypes binding (vie.py) with the same entry points.  Importing the package
does not load the library; `paper_1809_05334_gb300.vie.load()` does, and
fails loudly when it is missing.
"""
__all__ = ["vie"]
