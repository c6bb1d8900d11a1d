"""GB300-native two-site DMRG sigma engine (arXiv 2501.18263, Sec. 2.3-2.4).

The numerical path lives in the sm_103a shared library built from csrc/ and is
reached through the C ABI declared in include/dmrg_gb300.h; `binding` is the
thin ctypes layer with the same entry-point names.  `inputs` only draws seeded
synthetic inputs.  Importing this package does not load the CUDA library.
"""
__all__ = ["inputs", "binding"]
